// Runtime of libqfx: error state, launch accounting, kernel timing, plan tables on the
// device, and the executor behind qfx_amplitudes.
//
// Executor (Sec. III.A-III.B): the work is the list of items (slice, x1) for slices in
// [slice_begin, slice_end) and the n_batch bitstrings, slice-major.  As many items as
// the caller's workspace holds run together: fold + scale their site tensors, run every
// contraction step once for all of them (the item index is the GEMM's batch index), and
// add each item's result into out in FP64, in slice order.  No device memory is
// allocated here; all scratch lives in the caller's workspace, whose first
// table_bytes(p) bytes receive a copy of the plan's tables on every call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <new>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "ptx_async.cuh"
#include "qfx_internal.h"

namespace qfx {

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};

struct ProfRec {
  cudaEvent_t a, b;
  int step, variant, kind;
  double flops, bytes;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }
}  // namespace

qfx_status fail(qfx_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

qfx_status cuda_fail(int err, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString((cudaError_t)err);
  return QFX_ECUDA;
}

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

bool profile_on() { return g_prof_on; }

void profile_begin(void* stream, int* slot) {
  *slot = -1;
  if (!g_prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return;   // launches recorded into a graph are not timed here
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfRec r{};
  r.a = take_event();
  r.b = take_event();
  cudaEventRecord(r.a, (cudaStream_t)stream);
  g_prof.push_back(r);
  *slot = (int)g_prof.size() - 1;
}

void profile_end(void* stream, int slot, int step, int variant, int kind, double flops,
                 double bytes) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot >= (int)g_prof.size()) return;
  ProfRec& r = g_prof[slot];
  cudaEventRecord(r.b, (cudaStream_t)stream);
  r.step = step;
  r.variant = variant;
  r.kind = kind;
  r.flops = flops;
  r.bytes = bytes;
}

void build_table_image(qfx_plan* p) {
  std::vector<int64_t> partoff(p->sites.size());
  int64_t o = 0;
  for (size_t q = 0; q < p->sites.size(); ++q) {
    partoff[q] = o;
    o += adjoint_site_partials(p, p->sites[q]);
  }
  // the fold's float-float copy of the gate matrices: each FP64 entry d as hi = fl32(d)
  // and lo = fl32(d - hi) (d - hi is exact in FP64), so hi + lo holds d to ~48 bits
  std::vector<float> matsf(2 * p->mats.size());
  for (size_t j = 0; j < p->mats.size(); ++j) {
    const double d = p->mats[j];
    const float hi = static_cast<float>(d);
    matsf[2 * j] = hi;
    matsf[2 * j + 1] = static_cast<float>(d - static_cast<double>(hi));
  }
  const void* src[kTableRegions] = {p->sites.data(), p->events.data(), p->mats.data(),
                                    p->cut_dev.data(), p->open_perm.data(), p->gate_ev.data(),
                                    partoff.data(), matsf.data()};
  const size_t len[kTableRegions] = {p->sites.size() * sizeof(FoldSite), p->events.size() * sizeof(FoldEvent),
                                     p->mats.size() * sizeof(double), p->cut_dev.size() * sizeof(CutDev),
                                     p->open_perm.size() * sizeof(int32_t), p->gate_ev.size() * sizeof(int32_t),
                                     partoff.size() * sizeof(int64_t), matsf.size() * sizeof(float)};
  size_t total = 0;
  for (int r = 0; r < kTableRegions; ++r) {
    p->toffs[r] = total;
    total += align256(std::max<size_t>(1, len[r]));
  }
  // its own pages, so that page-locking it never touches another object's pages
  const uint64_t page = 4096;
  p->timg_bytes = total;
  p->timg_alloc = (total + page - 1) / page * page;
  void* mem = nullptr;
  if (posix_memalign(&mem, page, p->timg_alloc) != 0) throw std::bad_alloc();
  p->timg = (char*)mem;
  std::memset(p->timg, 0, p->timg_alloc);
  for (int r = 0; r < kTableRegions; ++r)
    if (len[r]) std::memcpy(p->timg + p->toffs[r], src[r], len[r]);
}

void free_table_image(qfx_plan* p) {
  if (!p->timg) return;
  if (p->timg_pinned) cudaHostUnregister(p->timg);
  free(p->timg);
  p->timg = nullptr;
}

qfx_status pin_tables(const qfx_plan* p) {
  std::lock_guard<std::mutex> lk(p->mu);
  if (p->timg_tried) return QFX_OK;
  p->timg_tried = true;
  cudaError_t e = cudaHostRegister(p->timg, p->timg_alloc, cudaHostRegisterPortable);
  if (e == cudaSuccess || e == cudaErrorHostMemoryAlreadyRegistered) {
    p->timg_pinned = e == cudaSuccess;
  } else {
    // the image stays pageable: copies from it remain correct (it lives as long as the
    // plan) but may make the host wait for the stream's earlier work
    (void)cudaGetLastError();
  }
  return QFX_OK;
}

qfx_status stage_tables(const qfx_plan* p, void* dst, void* stream, DeviceTables* out) {
  qfx_status s = pin_tables(p);
  if (s != QFX_OK) return s;
  cudaError_t e = cudaMemcpyAsync(dst, p->timg, p->timg_bytes, cudaMemcpyHostToDevice,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan tables -> workspace copy");
  *out = tables_at(dst, p->toffs);
  return QFX_OK;
}

DeviceTables tables_at(void* base, const size_t offs[kTableRegions]) {
  char* b = (char*)base;
  DeviceTables t;
  t.base = base;
  t.sites = (const FoldSite*)(b + offs[0]);
  t.events = (const FoldEvent*)(b + offs[1]);
  t.mats = (const double*)(b + offs[2]);
  t.cuts = (const CutDev*)(b + offs[3]);
  t.open_perm = (const int32_t*)(b + offs[4]);
  t.gate_ev = (const int32_t*)(b + offs[5]);
  t.partoff = (const int64_t*)(b + offs[6]);
  t.matsf = (const float*)(b + offs[7]);
  return t;
}

qfx_status check_amplitudes_args(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                 int64_t slice_begin, int64_t slice_end, const void* out) {
  if (!p || !x1 || !out) return fail(QFX_EINVAL, "qfx_amplitudes: NULL argument");
  if (n_batch < 1) return fail(QFX_EINVAL, "qfx_amplitudes: n_batch must be >= 1");
  if (slice_begin < 0 || slice_end > p->n_slices || slice_begin >= slice_end)
    return fail(QFX_EINVAL, "qfx_amplitudes: slice range outside [0, n_slices)");
  if (((uintptr_t)out & 15) != 0) return fail(QFX_EINVAL, "qfx_amplitudes: out not 16-byte aligned");
  return QFX_OK;
}

int64_t items_in_flight(const qfx_plan* p, size_t ws_bytes) {
  const uint64_t hdr = p->layout.header_per_item, ib = p->layout.item_bytes;
  int64_t G = (int64_t)(ws_bytes / (hdr + ib));
  while (G > 0 && align256((uint64_t)G * hdr) + (uint64_t)G * ib > ws_bytes) --G;
  return G;
}

// Contraction-tree plans: per group of items in flight, fold and scale their site
// tensors, then run the tree's nodes in order -- each operand's permute (one launch per
// item) and one batched GEMM launch over the items -- and add the root into `out`.
static qfx_status exec_tree(const qfx_plan* p, const DeviceTables& t, const uint64_t* x1,
                            int64_t n_batch, int64_t slice_begin, int64_t slice_end,
                            void* workspace, int64_t G, double* out, void* stream) {
  const Layout& L = p->layout;
  const uint64_t hdr = L.header_per_item, ib = L.item_bytes;
  const int64_t n_items = (slice_end - slice_begin) * n_batch;
  G = std::min<int64_t>({G, n_items, 65535});
  cudaStream_t st = (cudaStream_t)stream;
  const int n_open = (int)p->open_sites.size();
  int64_t max_site = 1;
  for (const auto& fs : p->sites) max_site = std::max(max_site, fs.size);
  char* hdr_base = (char*)workspace;
  char* items = hdr_base + align256((uint64_t)G * hdr);
  cudaError_t e = cudaMemsetAsync(out, 0, (size_t)(n_batch << n_open) * 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes: clearing out");
  for (int64_t item0 = 0; item0 < n_items; item0 += G) {
    const int g = (int)std::min<int64_t>(G, n_items - item0);
    e = cudaMemsetAsync(hdr_base, 0, (size_t)g * hdr, st);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes: clearing header");
    int slot;
    profile_begin(st, &slot);
    int err = launch_fold(t, p->n, max_site, (int)p->cut_dev.size(), x1, p->x1_words, n_batch,
                          slice_begin, item0, g, hdr_base, hdr, items, ib, L.sites, st);
    profile_end(st, slot, -1, 0, 1, 0.0, 0.0);
    if (err) return cuda_fail(err, "fold kernel");
    err = launch_scale(t, p->n, max_site, g, hdr_base, hdr, items, ib, L.sites, st);
    if (err) return cuda_fail(err, "scale kernel");
    for (size_t i = 0; i < p->tree.size(); ++i) {
      const TreeNode& nd = p->tree[i];
      for (int gi = 0; gi < g && (nd.permA || nd.permB); ++gi) {
        char* blk = items + (uint64_t)gi * ib;
        if (nd.permA) {
          profile_begin(st, &slot);
          err = launch_permute(blk + nd.offA, blk + nd.offA2, nd.rankA, nd.shapeA, nd.ordA, st);
          double el = 1;
          for (int a = 0; a < nd.rankA; ++a) el *= (double)nd.shapeA[a];
          profile_end(st, slot, (int)i, 0, 4, 0.0, 16.0 * el);
          if (err) return cuda_fail(err, "tree permute");
        }
        if (nd.permB) {
          profile_begin(st, &slot);
          err = launch_permute(blk + nd.offB, blk + nd.offB2, nd.rankB, nd.shapeB, nd.ordB, st);
          double el = 1;
          for (int a = 0; a < nd.rankB; ++a) el *= (double)nd.shapeB[a];
          profile_end(st, slot, (int)i, 0, 4, 0.0, 16.0 * el);
          if (err) return cuda_fail(err, "tree permute");
        }
      }
      profile_begin(st, &slot);
      if (nd.parts > 0) {
        // split K: chunk c's product into part[c] (the item's scratch), then the sum into C
        for (int gi = 0; gi < g && !err; ++gi) {
          char* blk = items + (uint64_t)gi * ib;
          err = launch_step(blk + nd.offA2, nd.chunk * nd.N, blk + nd.offB2, nd.chunk * nd.Sd,
                            blk + L.simage, nd.N * nd.Sd, 1, nd.chunk, nd.N, nd.NL, nd.Sd, nd.parts,
                            fill_variant(nd.variant, nd.N, nd.Sd, nd.parts), QFX_PREC_FP32_SIMT, st, 0);
        }
        if (!err)
          err = launch_reduce_parts(items + L.simage, (int64_t)(ib / 8), nd.parts, nd.N * nd.Sd,
                                    items + nd.offC, (int64_t)(ib / 8), g, st);
      }
      // a long contraction in chunks of nd.chunk rows of S and B (P = 1), each added into C
      for (int64_t k0 = 0; k0 < nd.K && !err && nd.parts == 0; k0 += nd.chunk) {
        const char* Sk = items + nd.offA2 + (uint64_t)(k0 * nd.N) * 8;
        const char* Bk = items + nd.offB2 + (uint64_t)(k0 * nd.Sd) * 8;
        if (nd.variant >= kVariantTcBf16)
          err = launch_step_tc(Sk, (int64_t)(ib / 8), Bk, (int64_t)(ib / 8), items + nd.offC,
                               (int64_t)(ib / 8), nd.P, nd.chunk, nd.N, nd.NL, nd.Sd, g, p->precision,
                               items + L.simage, (int64_t)ib, st, p->tc_flags | (k0 > 0 ? kTcBeta : 0));
        else
          err = launch_step(Sk, (int64_t)(ib / 8), Bk, (int64_t)(ib / 8), items + nd.offC,
                            (int64_t)(ib / 8), nd.P, nd.chunk, nd.N, nd.NL, nd.Sd, g,
                            fill_variant(nd.variant, nd.N, nd.P * nd.Sd, g), QFX_PREC_FP32_SIMT, st,
                            k0 > 0 ? 1 : 0);
      }
      profile_end(st, slot, (int)i, nd.variant, 0, nd.flops * g, nd.bytes * g);
      if (err) return cuda_fail(err, "contraction step kernel");
    }
    err = launch_accumulate(t, p->n, n_open, n_batch, item0, g, hdr_base, hdr, items, ib,
                            p->tree_final_off, out, st);
    if (err) return cuda_fail(err, "accumulate kernel");
  }
  return QFX_OK;
}

qfx_status exec_amplitudes(const qfx_plan* p, const DeviceTables& t, const uint64_t* x1,
                           int64_t n_batch, int64_t slice_begin, int64_t slice_end,
                           void* workspace, int64_t G, double* out, void* stream) {
  if (p->family == 1)
    return exec_tree(p, t, x1, n_batch, slice_begin, slice_end, workspace, G, out, stream);
  const Layout& L = p->layout;
  const uint64_t hdr = L.header_per_item, ib = L.item_bytes;
  const int64_t n_items = (slice_end - slice_begin) * n_batch;
  G = std::min<int64_t>({G, n_items, 65535});
  cudaStream_t st = (cudaStream_t)stream;
  const int n_open = (int)p->open_sites.size();
  const int n_sites = p->n;
  int64_t max_site = 1;
  for (const auto& fs : p->sites) max_site = std::max(max_site, fs.size);
  char* hdr_base = (char*)workspace;
  char* items = hdr_base + align256((uint64_t)G * hdr);
  const int nsteps = (int)p->steps.size();
  const uint64_t site0 = L.sites + (uint64_t)p->sites[p->steps[0].site].offset * 8;
  const uint64_t final_off = nsteps == 1 ? site0 : ((nsteps - 1) % 2 ? L.buf1 : L.buf0);

  cudaError_t e = cudaMemsetAsync(out, 0, (size_t)(n_batch << n_open) * 16, st);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes: clearing out");
  for (int64_t item0 = 0; item0 < n_items; item0 += G) {
    const int g = (int)std::min<int64_t>(G, n_items - item0);
    e = cudaMemsetAsync(hdr_base, 0, (size_t)g * hdr, st);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes: clearing header");
    int slot;
    profile_begin(st, &slot);
    int err = launch_fold(t, n_sites, max_site, (int)p->cut_dev.size(), x1, p->x1_words, n_batch,
                          slice_begin, item0, g, hdr_base, hdr, items, ib, L.sites, st);
    profile_end(st, slot, -1, 0, 1, 0.0, 0.0);
    if (err) return cuda_fail(err, "fold kernel");
    err = launch_scale(t, n_sites, max_site, g, hdr_base, hdr, items, ib, L.sites, st);
    if (err) return cuda_fail(err, "scale kernel");
    for (int i = 1; i < nsteps; ++i) {
      const Step& sp = p->steps[i];
      const char* S = items + L.sites + (uint64_t)p->sites[sp.site].offset * 8;
      const char* B = items + (i == 1 ? site0 : ((i - 1) % 2 ? L.buf1 : L.buf0));
      char* C = items + (i % 2 ? L.buf1 : L.buf0);
      profile_begin(st, &slot);
      if (sp.variant >= kVariantTcBf16)
        err = launch_step_tc(S, (int64_t)(ib / 8), B, (int64_t)(ib / 8), C, (int64_t)(ib / 8), sp.P,
                             sp.K, sp.N, sp.NL, sp.Sd, g, p->precision, items + L.simage,
                             (int64_t)ib, st, p->tc_flags);
      else
        err = launch_step(S, (int64_t)(ib / 8), B, (int64_t)(ib / 8), C, (int64_t)(ib / 8), sp.P,
                          sp.K, sp.N, sp.NL, sp.Sd, g, fill_variant(sp.variant, sp.N, sp.P * sp.Sd, g),
                          p->precision, st);
      profile_end(st, slot, i, sp.variant, 0, sp.flops * g, sp.bytes * g);
      if (err) return cuda_fail(err, "contraction step kernel");
    }
    err = launch_accumulate(t, n_sites, n_open, n_batch, item0, g, hdr_base, hdr, items, ib,
                            final_off, out, st);
    if (err) return cuda_fail(err, "accumulate kernel");
  }
  return QFX_OK;
}

}  // namespace qfx

using namespace qfx;

extern "C" qfx_status qfx_plan_upload(const qfx_plan* p) {
  if (!p) return fail(QFX_EINVAL, "qfx_plan_upload: NULL plan");
  return pin_tables(p);
}

extern "C" qfx_status qfx_amplitudes(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                     int64_t slice_begin, int64_t slice_end, void* workspace,
                                     size_t ws_bytes, double* out, void* stream) {
  qfx_status s = check_amplitudes_args(p, x1, n_batch, slice_begin, slice_end, out);
  if (s != QFX_OK) return s;
  if (!workspace) return fail(QFX_EINVAL, "qfx_amplitudes: NULL argument");
  if (((uintptr_t)workspace & 255) != 0) return fail(QFX_EINVAL, "qfx_amplitudes: workspace not 256-byte aligned");
  const uint64_t tb = table_bytes(p);
  const int64_t G = ws_bytes > tb ? items_in_flight(p, ws_bytes - tb) : 0;
  if (G < 1) return fail(QFX_ENOMEM, "qfx_amplitudes: workspace smaller than qfx_plan_stats.workspace_min");
  DeviceTables t;
  s = stage_tables(p, workspace, stream, &t);
  if (s != QFX_OK) return s;
  return exec_amplitudes(p, t, x1, n_batch, slice_begin, slice_end, (char*)workspace + tb, G, out,
                         stream);
}

// cuTensorMapEncodeTiled from the driver, looked up at run time (the library links only
// the static CUDA runtime, so it loads on machines without a driver).
PFN_cuTensorMapEncodeTiled_v12000 qfx::tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

extern "C" qfx_status qfx_sync(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_sync");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "qfx_sync");
  const int tc = tc_take_status();
  if (tc < 0) return fail(QFX_ECUDA, "qfx_sync: reading the tensor-core status word failed");
  if (tc > 0) return fail(QFX_ETIMEOUT, "qfx_sync: a tensor-core contraction step gave up waiting (bounded wait expired)");
  const int bt = batch_take_status();
  if (bt < 0) return fail(QFX_ECUDA, "qfx_sync: reading the batch status word failed");
  if (bt > 0) return fail(QFX_ETIMEOUT, "qfx_sync: the batch scheduler gave up a dependency wait (bounded wait expired)");
  const int pt = perm_take_status();
  if (pt < 0) return fail(QFX_ECUDA, "qfx_sync: reading the permute status word failed");
  if (pt > 0) return fail(QFX_ETIMEOUT, "qfx_sync: a permute copy did not arrive (bounded wait expired)");
  return QFX_OK;
}

extern "C" qfx_status qfx_tensor_peak(int32_t precision, int64_t mmas_per_sm, double* tflops, void* stream) {
  if (!tflops) return fail(QFX_EINVAL, "qfx_tensor_peak: NULL output");
  if (precision <= QFX_PREC_FP32_SIMT || precision > QFX_PREC_C3M_BF16X2)
    return fail(QFX_EINVAL, "qfx_tensor_peak: not a tensor-core precision");
  if (mmas_per_sm < 256) return fail(QFX_EINVAL, "qfx_tensor_peak: mmas_per_sm < 256");
  const int err = tc_probe(precision, mmas_per_sm, tflops, stream);
  if (err) return cuda_fail(err, "qfx_tensor_peak");
  const int tc = tc_take_status();
  if (tc != 0) return fail(QFX_ETIMEOUT, "qfx_tensor_peak: a bounded wait expired");
  return QFX_OK;
}

extern "C" uint64_t qfx_step_scratch_bytes(int64_t K, int64_t N, int32_t precision) {
  return tc_scratch_bytes(precision, K, N);
}

extern "C" qfx_status qfx_contract_step(const void* S, const void* B, void* C, int64_t P,
                                        int64_t K, int64_t N, int64_t NL, int64_t Sd,
                                        int32_t precision, int32_t variant, void* scratch,
                                        size_t scratch_bytes, void* stream) {
  if (!S || !B || !C) return fail(QFX_EINVAL, "qfx_contract_step: NULL pointer");
  if (P < 1 || K < 1 || N < 1 || NL < 1 || Sd < 1 || N % NL)
    return fail(QFX_EINVAL, "qfx_contract_step: need positive sizes and NL | N");
  if ((((uintptr_t)S) | ((uintptr_t)B) | ((uintptr_t)C)) & 15)
    return fail(QFX_EINVAL, "qfx_contract_step: pointers must be 16-byte aligned");
  if (precision < QFX_PREC_FP32_SIMT || precision > QFX_PREC_C3M_BF16X2)
    return fail(QFX_EINVAL, "qfx_contract_step: unknown precision");
  const bool tc = precision != QFX_PREC_FP32_SIMT &&
                  tc_eligible(precision, K, N, P * Sd, variant == 12 ? kTcFast : 0);
  if (tc) {
    if (!scratch || scratch_bytes < tc_scratch_bytes(precision, K, N) || ((uintptr_t)scratch & 255))
      return fail(QFX_ENOMEM, "qfx_contract_step: tensor-core steps need qfx_step_scratch_bytes() of 256-byte aligned scratch");
  }
  int flags = 0;
  if (variant == 99 && tc) { flags = kTcWithhold; variant = -1; }
  if (variant == 12 && tc) { flags = kTcFast; variant = -1; }
  if (variant == 13 && tc) { flags = kTcNoTma; variant = -1; }
  if (variant >= 0 && !simt_variant_valid(variant, 2))
    return fail(QFX_EINVAL, "qfx_contract_step: unknown variant");
  if (variant >= 0 && !simt_variant_valid(variant, Sd))
    return fail(QFX_EINVAL, "qfx_contract_step: variants 0-4 and 20-23 need an even Sd");
  int slot;
  profile_begin(stream, &slot);
  int v = variant < 0 ? fill_variant(pick_variant(N, Sd), N, P * Sd, 1) : variant;
  int err;
  if (tc) {
    v = precision == QFX_PREC_C3M_BF16X3 ? kVariantTcBf16
        : precision == QFX_PREC_C3M_BF16X2 ? kVariantTcBf16x2 : kVariantTcTf32;
    err = launch_step_tc(S, 0, B, 0, C, 0, P, K, N, NL, Sd, 1, precision, (char*)scratch, 0, stream,
                         flags);
  } else {
    err = launch_step(S, 0, B, 0, C, 0, P, K, N, NL, Sd, 1, v, precision, stream);
  }
  profile_end(stream, slot, -1, v, 0, 8.0 * P * K * N * Sd,
              8.0 * ((double)P * K * Sd + (double)K * N + (double)P * N * Sd));
  if (err) return cuda_fail(err, "qfx_contract_step");
  return QFX_OK;
}

extern "C" qfx_status qfx_permute(const void* in, void* out, int32_t rank, const int64_t* shape,
                                  const int32_t* perm, void* stream) {
  if (!in || !out || !shape || !perm) return fail(QFX_EINVAL, "qfx_permute: NULL argument");
  if (rank < 1 || rank > 10) return fail(QFX_EINVAL, "qfx_permute: rank must be 1..10");
  int seen = 0;
  for (int i = 0; i < rank; ++i) {
    if (perm[i] < 0 || perm[i] >= rank || (seen >> perm[i]) & 1)
      return fail(QFX_EINVAL, "qfx_permute: perm is not a permutation");
    seen |= 1 << perm[i];
    if (shape[i] < 0) return fail(QFX_EINVAL, "qfx_permute: negative extent");
  }
  int slot;
  profile_begin(stream, &slot);
  int err = launch_permute(in, out, rank, shape, perm, stream);
  double el = 1;
  for (int i = 0; i < rank; ++i) el *= (double)shape[i];
  profile_end(stream, slot, -1, 0, 4, 0.0, 16.0 * el);
  if (err) return cuda_fail(err, "qfx_permute");
  return QFX_OK;
}

extern "C" qfx_status qfx_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return QFX_OK;
}

extern "C" qfx_status qfx_profile_collect(qfx_kernel_time* out, int32_t max, int32_t* n) {
  if (!n) return fail(QFX_EINVAL, "qfx_profile_collect: NULL count");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int32_t k = 0;
  for (auto& r : g_prof) {
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_profile_collect");
    if (out && k < max) out[k] = qfx_kernel_time{r.step, r.variant, r.kind, ms, r.flops, r.bytes};
    ++k;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
  *n = k;
  return QFX_OK;
}

extern "C" uint64_t qfx_launch_count(void) { return g_launches.load(); }
extern "C" const char* qfx_last_error(void) { return g_err.c_str(); }
extern "C" const char* qfx_version(void) { return "qfx 0.1 (sm_103a)"; }
