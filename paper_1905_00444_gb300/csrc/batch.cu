// Batched execution of many (plan, slice, x1) work items of uneven shapes in ONE
// persistent kernel (Sec. III.A: slices are independent paths; Sec. III.B: x1 batches).
//
// The host expands a list of qfx_batch_item into work items and cuts each one's work
// into segments of independent tasks:
//   FOLD  (chunks of site elements: float-float time fold, per-site max) depends on the
//         previous occupant of the work item's workspace slot (its ACCUM);
//   SCALE (same chunks: power-of-two scale)                            on FOLD;
//   STEP i (output tiles of contraction step i, FP32 SIMT tile body)   on STEP i-1 / SCALE;
//   ACCUM (FP64 2^E-scaled add into the output row)                    on the last STEP and
//         on the ACCUM of the previous slice of the same output row (fixed FP64 order).
// Segments are listed round by round (a round = one work item per slot), phase by phase,
// so every dependency points to an earlier task.  CTAs take tasks in that order from a
// global counter; before a task, thread 0 waits (acquire, bounded) until the segments it
// depends on have counted all their tiles, and after it, releases one count.  Because a
// task is only taken by a running CTA and only waits on earlier tasks, the queue always
// makes progress; the bound (5 s per wait) only guards against a bug, and on expiry the
// kernel sets an abort flag that every CTA sees, records QFX_ETIMEOUT and exits.
// qfx_batch_prepare uploads the schedule once; qfx_batch_run is two memsets and one
// launch, with no host synchronisation or allocation, so it can be captured in a graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "cgemm_tile.cuh"
#include "fold_element.cuh"
#include "qfx_internal.h"

namespace qfx {

__device__ unsigned int g_batch_status = 0;

namespace {

constexpr int kT = 256;
constexpr int64_t kFoldChunk = 2048;
constexpr unsigned long long kDepWaitNs = 5000000000ull;
enum Phase : int32_t { PH_FOLD = 0, PH_SCALE = 1, PH_ACCUM = 2, PH_STEP0 = 2 };  // step i -> 2 + i

struct StepDev {
  int32_t site, variant;
  int64_t P, K, N, NL, Sd;
};

struct PlanDev {
  DeviceTables t;
  const StepDev* steps;
  const int32_t* chunk_site;
  const int64_t* chunk_start;
  int32_t n_sites, n_steps, n_open, n_cuts, n_chunks, pad;
  uint64_t buf0, buf1, sites, final_off, site0_off;
};

struct WorkDev {
  int32_t plan, slot;
  int64_t b, sid;
  const uint64_t* x1;     // this work item's bitstring (x1_words words)
  double* out;            // this work item's output row
  int32_t first, pad;     // first slice of the row: assign instead of add
};

struct SegDev {
  int64_t first_task;
  int32_t work, phase, tiles;
  int32_t dep[2], need[2];
};

struct BatchArgs {
  const SegDev* segs;
  int32_t n_segs;
  int64_t n_tasks;
  const WorkDev* work;
  const PlanDev* plans;
  int32_t* done;
  unsigned long long* head;
  int32_t* abort;
  char* hdrs;             // slot headers: maxabs[64] (u32) + exps[64] (i32) each
  char* blocks;           // slot item blocks
  uint64_t hdr_bytes, block_bytes;
  unsigned long long wait_ns;   // limit of each dependency wait
};

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void add_release(int32_t* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ void run_step_tile(const simt::StepArgs& a, int variant, int64_t tile, float4* smem) {
  switch (variant) {
#define QFX_CASE(V, BM, BJ, TM, TJ, KM, ST) \
  case V: simt::cgemm_tile<BM, BJ, TM, TJ, KM, ST>(a, tile, 0, smem); break;
    QFX_SIMT_VARIANTS(QFX_CASE)
#undef QFX_CASE
    default: break;
  }
}

__global__ void __launch_bounds__(kT, 1) batch_kernel(const BatchArgs a) {
  extern __shared__ float4 smem[];
  __shared__ long long s_task;
  __shared__ int s_seg, s_go;
  __shared__ float s_max[kT / 32];
  const int tid = threadIdx.x;
  // thread 0 keeps the next task index in flight and the last segment it found: task
  // indices handed to one CTA only grow, so the next segment is found by galloping
  // forward from the previous one (a few dependent loads instead of a full search).
  long long next_t = 0;
  int last = 0;
  if (tid == 0) next_t = (long long)atomicAdd(a.head, 1ull);
  for (;;) {
    if (tid == 0) {
      s_go = 0;
      const long long t = next_t;
      if (t < a.n_tasks && !*(volatile int32_t*)a.abort) {
        next_t = (long long)atomicAdd(a.head, 1ull);
        int lo = last, step = 1;
        while (lo + step < a.n_segs && a.segs[lo + step].first_task <= t) { lo += step; step <<= 1; }
        int hi = min(a.n_segs - 1, lo + step);
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.segs[mid].first_task <= t) lo = mid; else hi = mid - 1;
        }
        last = lo;
        s_task = t;
        s_seg = lo;
        s_go = 1;
        const SegDev sg = a.segs[lo];
        for (int d = 0; d < 2 && s_go; ++d) {
          if (sg.dep[d] < 0) continue;
          if (ld_acquire(a.done + sg.dep[d]) >= sg.need[d]) continue;
          const unsigned long long deadline = gtimer() + a.wait_ns;
          while (ld_acquire(a.done + sg.dep[d]) < sg.need[d]) {
            if (*(volatile int32_t*)a.abort) { s_go = 0; break; }
            if (gtimer() > deadline) {
              atomicExch(a.abort, 1);
              atomicOr(&g_batch_status, 1u);
              s_go = 0;
              break;
            }
            __nanosleep(64);
          }
        }
      }
    }
    __syncthreads();
    if (!s_go) break;
    const SegDev sg = a.segs[s_seg];
    const int64_t tile = s_task - sg.first_task;
    const WorkDev w = a.work[sg.work];
    const PlanDev pl = a.plans[w.plan];
    char* hdr = a.hdrs + (uint64_t)w.slot * a.hdr_bytes;
    unsigned* maxabs = reinterpret_cast<unsigned*>(hdr);
    int* exps = reinterpret_cast<int*>(hdr) + kMaxSites;
    char* blk = a.blocks + (uint64_t)w.slot * a.block_bytes;
    float2* sites = reinterpret_cast<float2*>(blk + pl.sites);

    if (sg.phase == PH_FOLD || sg.phase == PH_SCALE) {
      const int s = pl.chunk_site[tile];
      const int64_t start = pl.chunk_start[tile];
      const FoldSite st = pl.t.sites[s];
      const int64_t end = min(st.size, start + kFoldChunk);
      float2* T = sites + st.offset;
      if (sg.phase == PH_FOLD) {
        float mx = 0.f;
        for (int64_t i = start + tid; i < end; i += kT) {
          const float2 v = foldk::fold_element(st, pl.t.events, pl.t.matsf, pl.t.cuts, pl.n_cuts,
                                               w.x1, w.sid, i);
          T[i] = v;
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
        if ((tid & 31) == 0) s_max[tid >> 5] = __uint_as_float(bits);
        __syncthreads();
        if (tid == 0) {
          float m = 0.f;
          for (int q = 0; q < kT / 32; ++q) m = fmaxf(m, s_max[q]);
          if (m > 0.f) atomicMax(maxabs + s, __float_as_uint(m));
        }
      } else {
        const float m = __uint_as_float(((volatile unsigned*)maxabs)[s]);
        int e = 0;
        if (m > 0.f) frexpf(m, &e);
        if (start == 0 && tid == 0) exps[s] = e;
        if (e != 0) {
          const float sc = ldexpf(1.0f, -e);
          for (int64_t i = start + tid; i < end; i += kT) {
            float2 v = T[i];
            v.x *= sc;
            v.y *= sc;
            T[i] = v;
          }
        }
      }
    } else if (sg.phase == PH_ACCUM) {
      int E = 0;
      for (int q = 0; q < pl.n_sites; ++q) E += ((volatile int*)exps)[q];
      const float2* fin = reinterpret_cast<const float2*>(blk + pl.final_off);
      const int64_t per = int64_t(1) << pl.n_open;
      for (int64_t o = tid; o < per; o += kT) {
        int64_t f = 0;
        for (int i = 0; i < pl.n_open; ++i) f |= ((o >> i) & 1) << pl.t.open_perm[i];
        const float2 c = fin[f];
        double re = ldexp((double)c.x, E), im = ldexp((double)c.y, E);
        if (!w.first) { re += w.out[2 * o]; im += w.out[2 * o + 1]; }
        w.out[2 * o] = re;
        w.out[2 * o + 1] = im;
      }
      // the slot's next occupant starts its per-site maxima from zero
      if (tid < pl.n_sites) maxabs[tid] = 0u;
    } else {
      const int i = sg.phase - PH_STEP0;
      const StepDev sp = pl.steps[i];
      const FoldSite st = pl.t.sites[sp.site];
      simt::StepArgs sa{};
      sa.S = sites + st.offset;
      sa.B = reinterpret_cast<const float2*>(blk + (i == 1 ? pl.site0_off : ((i - 1) % 2 ? pl.buf1 : pl.buf0)));
      sa.C = reinterpret_cast<float2*>(blk + (i % 2 ? pl.buf1 : pl.buf0));
      sa.P = sp.P; sa.K = sp.K; sa.N = sp.N; sa.NL = sp.NL; sa.Sd = sp.Sd; sa.J = sp.P * sp.Sd;
      run_step_tile(sa, sp.variant, tile, smem);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      add_release(a.done + s_seg, 1);
    }
  }
}

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

constexpr int64_t kGraphLanes = 16;

}  // namespace

// Workspace of one graph lane: the header and block of one work item of the largest plan.
uint64_t graph_lane_bytes(const qfx_batch_item* items, int32_t n_items) {
  uint64_t lane = 0;
  for (int i = 0; i < n_items; ++i) {
    const qfx_plan* p = items[i].plan;
    lane = std::max<uint64_t>(lane, a256(p->layout.header_per_item) + p->layout.item_bytes);
  }
  return a256(lane);
}

namespace {

size_t batch_smem() {
  size_t m = 0;
#define QFX_SZ(V, BM, BJ, TM, TJ, KM, ST) m = std::max(m, simt::Cfg<BM, BJ, TM, TJ, KM, ST>::SMEM);
  QFX_SIMT_VARIANTS(QFX_SZ)
#undef QFX_SZ
  return m;
}

int64_t step_tiles(int variant, int64_t N, int64_t J) {
  int bm = 128, bj = 128;
  switch (variant) {
#define QFX_T(V, BM, BJ, TM, TJ, KM, ST) case V: bm = BM; bj = BJ; break;
    QFX_SIMT_VARIANTS(QFX_T)
#undef QFX_T
    default: break;
  }
  return ((N + bm - 1) / bm) * ((J + bj - 1) / bj);
}

}  // namespace

int batch_take_status() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_batch_status, sizeof(v)) != cudaSuccess) return -1;
  if (v) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_batch_status, &z, sizeof(z));
  }
  return (int)v;
}

}  // namespace qfx

struct qfx_batch {
  std::vector<char> host;          // uploaded image (kept alive for the async copy)
  qfx::BatchArgs args{};
  void* control = nullptr;         // head, abort, done[] (cleared by every run)
  size_t control_bytes = 0;
  size_t hdrs_bytes = 0;
  int grid = 0;
  size_t smem = 0;
  int64_t n_work = 0, slots = 0;
  // batches with tensor-core or large items: one CUDA graph of per-item launch sequences
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  qfx_batch* sub = nullptr;        // persistent sub-batch of the small items, run inside the graph
  ~qfx_batch() {
    delete sub;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

using namespace qfx;

// Whether an FP32 work item runs as its own launch sequence in a batch's graph: its
// largest step has at least kBigTiles output tiles, so the step kernels fill the GPU many
// times over and launch overhead is negligible, while the same tiles run slower inside the
// persistent kernel (measured: 48.2 against 41.6 TFLOP/s on the mixed-grid batch).
constexpr int64_t kBigTiles = 512;
bool item_is_big(const qfx_plan* p) {
  if (p->family == 1) return true;   // contraction trees run through the launch path only
  int64_t most = 0;
  for (size_t i = 1; i < p->steps.size(); ++i) {
    const Step& sp = p->steps[i];
    const int v = sp.variant >= kVariantTcBf16 ? pick_variant(sp.N, sp.Sd) : sp.variant;
    most = std::max(most, step_tiles(v, sp.N, sp.P * sp.Sd));
  }
  return most >= kBigTiles;
}

// Whether a work item runs as its own launch sequence in a batch's graph rather than inside
// the persistent kernel: its plan has a step on the tensor cores (that tile has its own
// warp roles, TMEM and barrier rings, and is itself persistent over a step's tiles), or it
// is big (above).  Split-precision plans whose steps all resolve to FP32 tiles (step
// shapes the tensor-core tile does not take: K or N below 16, fewer than 128 columns, as
// in 4x4x(1+16+1) with bond dimension 4) run in the persistent kernel like FP32 plans: the
// FP32 tile ignores the plan's precision.
bool item_runs_launches(const qfx_plan* p) {
  for (const auto& sp : p->steps)
    if (sp.variant >= kVariantTcBf16) return true;
  return item_is_big(p);
}

static qfx_status prepare_persistent(const qfx_batch_item* items, int32_t n_items,
                                     const std::map<const qfx_plan*, const DeviceTables*>& tabmap,
                                     void* workspace, size_t ws_bytes, qfx_batch** out, void* stream);

static uint64_t qfx_batch_workspace_bytes_nt(const qfx_batch_item* items, int32_t n_items, int64_t slots);

// Workspace of the persistent sub-batch of a graph batch (its small items, 16 slots).
constexpr int64_t kSubSlots = 16;
static uint64_t sub_bytes(const std::vector<qfx_batch_item>& small) {
  return small.empty() ? 0 : a256(qfx_batch_workspace_bytes_nt(small.data(), (int32_t)small.size(), kSubSlots));
}

// Graph executor.  Every item's ordinary launch sequence (qfx_amplitudes' fold, scale,
// steps, accumulation; one work item in flight) is recorded on one of `lanes` streams
// forked from a capture stream, each lane with its own workspace slot, and the lanes join
// again: one CUDA graph, replayed by qfx_batch_run.  Items on different lanes overlap; an
// item's own launches keep their order.  Items with tensor-core steps and large items run
// this way; the small FP32-tile items (`small`) run in one persistent launch recorded on a
// lane of its own.
static qfx_status prepare_graph(const qfx_batch_item* items, int32_t n_items,
                                const std::vector<qfx_batch_item>& small,
                                const std::map<const qfx_plan*, const DeviceTables*>& tabmap,
                                void* workspace, size_t ws_bytes, qfx_batch** out, void* stream) {
  const uint64_t lane = graph_lane_bytes(items, n_items);
  const uint64_t sub_ws = sub_bytes(small);
  if (ws_bytes < sub_ws) return fail(QFX_ENOMEM, "qfx_batch_prepare: workspace smaller than the small items' share");
  int64_t n_work = 0;
  for (int i = 0; i < n_items; ++i) n_work += (items[i].slice_end - items[i].slice_begin) * items[i].n_batch;
  const int64_t lanes = std::min<int64_t>({kGraphLanes, (int64_t)((ws_bytes - sub_ws) / lane), (int64_t)n_items});
  if (lanes < 1) return fail(QFX_ENOMEM, "qfx_batch_prepare: workspace smaller than one work item");
  // kernel attributes are set before the capture (a captured launch must not be the first)
  int err = tc_prepare_attributes();
  if (!err) err = simt_prepare_attributes();
  if (err) return cuda_fail(err, "qfx_batch_prepare: kernel attributes");
  auto* B = new qfx_batch;
  std::unique_ptr<qfx_batch> guard(B);
  if (!small.empty()) {   // uploads its schedule now, before the capture
    qfx_status s = prepare_persistent(small.data(), (int32_t)small.size(), tabmap, workspace, sub_ws,
                                      &B->sub, stream);
    if (s != QFX_OK) return s;
  }
  char* lanes_base = (char*)workspace + sub_ws;
  const int64_t n_streams = lanes + (small.empty() ? 0 : 1);
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> ls((size_t)n_streams, nullptr);
  std::vector<cudaEvent_t> ev((size_t)n_streams + 1, nullptr);
  auto release = [&]() {
    for (auto& x : ls) if (x) cudaStreamDestroy(x);
    for (auto& x : ev) if (x) cudaEventDestroy(x);
    if (cap) cudaStreamDestroy(cap);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (int64_t l = 0; l < n_streams && e == cudaSuccess; ++l) e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking);
  for (size_t l = 0; l < ev.size() && e == cudaSuccess; ++l) e = cudaEventCreateWithFlags(&ev[l], cudaEventDisableTiming);
  if (e != cudaSuccess) { release(); return cuda_fail(e, "qfx_batch_prepare: streams"); }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { release(); return cuda_fail(e, "qfx_batch_prepare: begin capture"); }
  qfx_status st = QFX_OK;
  e = cudaEventRecord(ev[n_streams], cap);
  for (int64_t l = 0; l < n_streams && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(ls[l], ev[n_streams], 0);
  if (e != cudaSuccess) st = cuda_fail(e, "qfx_batch_prepare: fork");
  if (st == QFX_OK && B->sub) st = qfx_batch_run(B->sub, ls[lanes]);
  for (int i = 0; i < n_items && st == QFX_OK; ++i) {
    const qfx_batch_item& it = items[i];
    const int64_t l = i % lanes;
    st = exec_amplitudes(it.plan, *tabmap.at(it.plan), it.x1, it.n_batch, it.slice_begin,
                         it.slice_end, lanes_base + l * lane, 1, it.out, ls[l]);
  }
  for (int64_t l = 0; l < n_streams && st == QFX_OK; ++l) {
    e = cudaEventRecord(ev[l], ls[l]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[l], 0);
    if (e != cudaSuccess) st = cuda_fail(e, "qfx_batch_prepare: join");
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);   // ends the capture in every case
  release();
  if (st != QFX_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "qfx_batch_prepare: capture"); }
  B->graph = g;
  e = cudaGraphInstantiate(&B->exec, g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: graph instantiation");
  size_t nn = 0;
  e = cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: graph nodes");
  int64_t kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  B->graph_kernels = kernels;
  B->n_work = n_work + (B->sub ? B->sub->n_work : 0);
  B->slots = lanes;
  B->args.n_tasks = (int64_t)nn;
  *out = guard.release();
  return QFX_OK;
}

// The persistent scheduler: one launch runs every work item of `items` (FP32 plans).
static qfx_status prepare_persistent(const qfx_batch_item* items, int32_t n_items,
                                     const std::map<const qfx_plan*, const DeviceTables*>& tabmap,
                                     void* workspace, size_t ws_bytes, qfx_batch** out, void* stream) {
  try {
    std::map<const qfx_plan*, int> plan_ix;
    std::vector<const qfx_plan*> plans;
    std::vector<const DeviceTables*> tabs;
    for (int i = 0; i < n_items; ++i)
      if (!plan_ix.count(items[i].plan)) {
        plan_ix[items[i].plan] = (int)plans.size();
        plans.push_back(items[i].plan);
        tabs.push_back(tabmap.at(items[i].plan));
      }
    // work items, slice-major within each batch item
    struct W { int plan; int64_t b, sid; const qfx_batch_item* it; bool first; };
    std::vector<W> work;
    for (int i = 0; i < n_items; ++i) {
      const qfx_batch_item& it = items[i];
      for (int64_t s = it.slice_begin; s < it.slice_end; ++s)
        for (int64_t b = 0; b < it.n_batch; ++b) work.push_back({plan_ix[it.plan], b, s, &it, s == it.slice_begin});
    }
    const int64_t NW = (int64_t)work.size();
    // per-plan device tables: steps and fold chunks
    uint64_t block = 0;
    std::vector<std::vector<StepDev>> psteps(plans.size());
    std::vector<std::vector<int32_t>> pcs(plans.size());
    std::vector<std::vector<int64_t>> pcst(plans.size());
    for (size_t k = 0; k < plans.size(); ++k) {
      const qfx_plan* p = plans[k];
      block = std::max<uint64_t>(block, p->layout.item_bytes);
      for (const auto& sp : p->steps) {
        int v = sp.variant >= 10 ? pick_variant(sp.N, sp.Sd) : sp.variant;   // FP32 tiles only
        psteps[k].push_back({sp.site, v, sp.P, sp.K, sp.N, sp.NL, sp.Sd});
      }
      for (int q = 0; q < p->n; ++q)
        for (int64_t st = 0; st < p->sites[q].size; st += kFoldChunk) {
          pcs[k].push_back(q);
          pcst[k].push_back(st);
        }
      if (p->n > kMaxSites) return fail(QFX_EINVAL, "qfx_batch_prepare: too many sites");
    }
    // segments
    std::vector<SegDev> segs;
    std::vector<int32_t> accum_seg(NW, -1), last_seg(NW, -1), scale_seg(NW, -1);
    // slots from the workspace size
    const uint64_t hdr_b = a256(kMaxSites * 8), blk_b = a256(block);
    int64_t segs_est = 0;
    for (const auto& w : work) segs_est += (int64_t)plans[w.plan]->steps.size() + 3;
    // image layout: [control][segs][work][plans][per-plan steps/chunks][hdrs][blocks]
    const uint64_t control_b = a256(64 + (uint64_t)segs_est * 4);
    uint64_t tab_b = a256((uint64_t)segs_est * sizeof(SegDev)) + a256((uint64_t)NW * sizeof(WorkDev)) +
                     a256(plans.size() * sizeof(PlanDev));
    for (size_t k = 0; k < plans.size(); ++k)
      tab_b += a256(psteps[k].size() * sizeof(StepDev)) + a256(pcs[k].size() * 4) + a256(pcst[k].size() * 8);
    if (ws_bytes < control_b + tab_b + hdr_b + blk_b)
      return fail(QFX_ENOMEM, "qfx_batch_prepare: workspace too small for one slot");
    int64_t G = (int64_t)((ws_bytes - control_b - tab_b) / (hdr_b + blk_b));
    G = std::max<int64_t>(1, std::min(G, NW));
    std::map<std::pair<const qfx_batch_item*, int64_t>, int32_t> prev_row_accum;
    int64_t task = 0;
    auto add = [&](int32_t w, int32_t ph, int64_t tiles, int32_t d0, int32_t n0, int32_t d1, int32_t n1) {
      SegDev s{};
      s.first_task = task;
      s.work = w;
      s.phase = ph;
      s.tiles = (int32_t)tiles;
      s.dep[0] = d0; s.need[0] = n0;
      s.dep[1] = d1; s.need[1] = n1;
      segs.push_back(s);
      task += tiles;
      return (int32_t)segs.size() - 1;
    };
    for (int64_t r0 = 0; r0 < NW; r0 += G) {
      const int64_t r1 = std::min(NW, r0 + G);
      std::vector<int32_t> fold_seg(r1 - r0);
      for (int64_t w = r0; w < r1; ++w) {
        const int64_t prev = w - G;
        const int32_t d = prev >= 0 ? accum_seg[prev] : -1;
        fold_seg[w - r0] = add((int32_t)w, PH_FOLD, (int64_t)pcs[work[w].plan].size(), d, 1, -1, 0);
      }
      for (int64_t w = r0; w < r1; ++w) {
        const int32_t f = fold_seg[w - r0];
        scale_seg[w] = add((int32_t)w, PH_SCALE, segs[f].tiles, f, segs[f].tiles, -1, 0);
        last_seg[w] = scale_seg[w];
      }
      int max_steps = 0;
      for (int64_t w = r0; w < r1; ++w) max_steps = std::max(max_steps, (int)plans[work[w].plan]->steps.size());
      for (int i = 1; i < max_steps; ++i)
        for (int64_t w = r0; w < r1; ++w) {
          const auto& ps = psteps[work[w].plan];
          if (i >= (int)ps.size()) continue;
          const int64_t tiles = step_tiles(ps[i].variant, ps[i].N, ps[i].P * ps[i].Sd);
          const int32_t d = last_seg[w];
          last_seg[w] = add((int32_t)w, PH_STEP0 + i, tiles, d, segs[d].tiles, -1, 0);
        }
      for (int64_t w = r0; w < r1; ++w) {
        const auto key = std::make_pair(work[w].it, work[w].b);
        const int32_t prow = work[w].first ? -1 : prev_row_accum[key];
        const int32_t d = last_seg[w];
        accum_seg[w] = add((int32_t)w, PH_ACCUM, 1, d, segs[d].tiles, prow, prow >= 0 ? 1 : 0);
        prev_row_accum[key] = accum_seg[w];
      }
    }
    // build the image
    auto* B = new qfx_batch;
    std::unique_ptr<qfx_batch> guard(B);
    char* dev = (char*)workspace;
    const uint64_t control_bytes = a256(64 + segs.size() * 4);
    uint64_t o = control_bytes;
    const uint64_t o_segs = o; o += a256(segs.size() * sizeof(SegDev));
    const uint64_t o_work = o; o += a256((uint64_t)NW * sizeof(WorkDev));
    const uint64_t o_plans = o; o += a256(plans.size() * sizeof(PlanDev));
    std::vector<uint64_t> o_steps(plans.size()), o_cs(plans.size()), o_cst(plans.size());
    for (size_t k = 0; k < plans.size(); ++k) {
      o_steps[k] = o; o += a256(psteps[k].size() * sizeof(StepDev));
      o_cs[k] = o; o += a256(pcs[k].size() * 4);
      o_cst[k] = o; o += a256(pcst[k].size() * 8);
    }
    const uint64_t image_end = o;
    const uint64_t o_hdrs = o; o += (uint64_t)G * hdr_b;
    const uint64_t o_blocks = o; o += (uint64_t)G * blk_b;
    if (o > ws_bytes) return fail(QFX_ENOMEM, "qfx_batch_prepare: workspace layout overflow");
    B->host.assign(image_end - control_bytes, 0);
    auto at = [&](uint64_t ws_off) { return B->host.data() + (ws_off - control_bytes); };
    std::memcpy(at(o_segs), segs.data(), segs.size() * sizeof(SegDev));
    std::vector<WorkDev> wd(NW);
    for (int64_t w = 0; w < NW; ++w) {
      const qfx_plan* p = plans[work[w].plan];
      const int64_t per = int64_t(1) << p->open_sites.size();
      wd[w] = WorkDev{work[w].plan, (int32_t)(w % G), work[w].b, work[w].sid,
                      work[w].it->x1 + work[w].b * p->x1_words,
                      work[w].it->out + 2 * work[w].b * per, work[w].first ? 1 : 0, 0};
    }
    std::memcpy(at(o_work), wd.data(), wd.size() * sizeof(WorkDev));
    std::vector<PlanDev> pd(plans.size());
    for (size_t k = 0; k < plans.size(); ++k) {
      const qfx_plan* p = plans[k];
      PlanDev d{};
      d.t = *tabs[k];
      d.steps = (const StepDev*)(dev + o_steps[k]);
      d.chunk_site = (const int32_t*)(dev + o_cs[k]);
      d.chunk_start = (const int64_t*)(dev + o_cst[k]);
      d.n_sites = p->n;
      d.n_steps = (int32_t)p->steps.size();
      d.n_open = (int32_t)p->open_sites.size();
      d.n_cuts = (int32_t)p->cut_dev.size();
      d.n_chunks = (int32_t)pcs[k].size();
      d.buf0 = p->layout.buf0;
      d.buf1 = p->layout.buf1;
      d.sites = p->layout.sites;
      d.site0_off = p->layout.sites + (uint64_t)p->sites[p->steps[0].site].offset * 8;
      const int ns = (int)p->steps.size();
      d.final_off = ns == 1 ? d.site0_off : ((ns - 1) % 2 ? p->layout.buf1 : p->layout.buf0);
      pd[k] = d;
      std::memcpy(at(o_steps[k]), psteps[k].data(), psteps[k].size() * sizeof(StepDev));
      std::memcpy(at(o_cs[k]), pcs[k].data(), pcs[k].size() * 4);
      std::memcpy(at(o_cst[k]), pcst[k].data(), pcst[k].size() * 8);
    }
    std::memcpy(at(o_plans), pd.data(), pd.size() * sizeof(PlanDev));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dev + control_bytes, B->host.data(), B->host.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: schedule upload");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: schedule upload");
    BatchArgs& A = B->args;
    A.segs = (const SegDev*)(dev + o_segs);
    A.n_segs = (int32_t)segs.size();
    A.n_tasks = task;
    A.work = (const WorkDev*)(dev + o_work);
    A.plans = (const PlanDev*)(dev + o_plans);
    A.head = (unsigned long long*)dev;
    A.abort = (int32_t*)(dev + 8);
    A.done = (int32_t*)(dev + 64);
    A.hdrs = dev + o_hdrs;
    A.blocks = dev + o_blocks;
    A.hdr_bytes = hdr_b;
    A.block_bytes = blk_b;
    A.wait_ns = kDepWaitNs;
    B->control = dev;
    B->control_bytes = control_bytes;
    B->hdrs_bytes = (uint64_t)G * hdr_b;
    B->smem = batch_smem();
    B->n_work = NW;
    B->slots = G;
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: smem attribute");
    int occ = 0, dev_id = 0, sms = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kT, B->smem);
    if (e != cudaSuccess || occ < 1) return fail(QFX_ECUDA, "qfx_batch_prepare: kernel does not fit an SM");
    B->grid = (int)std::min<int64_t>((int64_t)sms * occ, std::max<int64_t>(1, task));
    *out = guard.release();
    return QFX_OK;
  } catch (const std::exception& ex) {
    return fail(QFX_EINVAL, std::string("qfx_batch_prepare: ") + ex.what());
  }
}

// Workspace of a persistent batch of `items` with `slots` items in flight (no plan tables).
static uint64_t qfx_batch_workspace_bytes_nt(const qfx_batch_item* items, int32_t n_items, int64_t slots) {
  uint64_t block = 0;
  int64_t segs_est = 0, work = 0;
  for (int i = 0; i < n_items; ++i) {
    const qfx_plan* p = items[i].plan;
    block = std::max<uint64_t>(block, p->layout.item_bytes);
    const int64_t w = (items[i].slice_end - items[i].slice_begin) * items[i].n_batch;
    work += w;
    segs_est += w * ((int64_t)p->steps.size() + 3);
  }
  const uint64_t tables = a256((uint64_t)segs_est * sizeof(SegDev)) + a256((uint64_t)work * sizeof(WorkDev)) +
                          (uint64_t)n_items * (64 * 1024) + (1u << 20);
  const uint64_t control = a256(64 + (uint64_t)segs_est * 4);
  return control + tables + (uint64_t)slots * (a256(kMaxSites * 8) + a256(block));
}

extern "C" uint64_t qfx_batch_workspace_bytes(const qfx_batch_item* items, int32_t n_items,
                                              int64_t slots) {
  if (!items || n_items < 1 || slots < 1) return 0;
  std::set<const qfx_plan*> distinct;
  uint64_t tab = 0;   // one copy of each distinct plan's tables
  for (int i = 0; i < n_items; ++i) {
    if (!items[i].plan) return 0;
    if (distinct.insert(items[i].plan).second) tab += qfx::table_bytes(items[i].plan);
  }
  std::vector<qfx_batch_item> big, small;
  for (int i = 0; i < n_items; ++i) (item_runs_launches(items[i].plan) ? big : small).push_back(items[i]);
  if (!big.empty())
    return tab + sub_bytes(small) + (uint64_t)slots * qfx::graph_lane_bytes(big.data(), (int32_t)big.size());
  return tab + qfx_batch_workspace_bytes_nt(items, n_items, slots);
}

extern "C" qfx_status qfx_batch_prepare(const qfx_batch_item* items, int32_t n_items, void* workspace,
                                        size_t ws_bytes, qfx_batch** out, void* stream) {
  if (!items || n_items < 1 || !workspace || !out) return fail(QFX_EINVAL, "qfx_batch_prepare: bad arguments");
  *out = nullptr;
  if ((uintptr_t)workspace & 255) return fail(QFX_EINVAL, "qfx_batch_prepare: workspace not 256-byte aligned");
  try {
    std::map<const qfx_plan*, int> plan_ix;
    std::vector<const qfx_plan*> plans;
    for (int i = 0; i < n_items; ++i) {
      const qfx_batch_item& it = items[i];
      qfx_status s = check_amplitudes_args(it.plan, it.x1, it.n_batch, it.slice_begin, it.slice_end, it.out);
      if (s != QFX_OK) return s;
      if (!plan_ix.count(it.plan)) {
        plan_ix[it.plan] = (int)plans.size();
        plans.push_back(it.plan);
      }
    }
    // plan tables: one copy per distinct plan at the start of the workspace, uploaded
    // here (synchronously, before any capture); the schedule lives after them
    std::vector<DeviceTables> tab_store(plans.size());
    std::vector<const DeviceTables*> tabs;
    {
      uint64_t o = 0;
      cudaStream_t st = (cudaStream_t)stream;
      for (size_t k = 0; k < plans.size(); ++k) {
        if (o + table_bytes(plans[k]) > ws_bytes) return fail(QFX_ENOMEM, "qfx_batch_prepare: workspace smaller than the plans' tables");
        qfx_status s = stage_tables(plans[k], (char*)workspace + o, stream, &tab_store[k]);
        if (s != QFX_OK) return s;
        tabs.push_back(&tab_store[k]);
        o += table_bytes(plans[k]);
      }
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_prepare: plan tables");
      workspace = (char*)workspace + o;
      ws_bytes -= o;
    }
    std::map<const qfx_plan*, const DeviceTables*> tabmap;
    for (size_t k = 0; k < plans.size(); ++k) tabmap[plans[k]] = tabs[k];
    // Items with tensor-core steps, and items whose steps fill the GPU many times over, run
    // as their own launch sequences inside one graph (the tensor-core tile cannot run as a
    // task of the persistent kernel, large FP32 tiles run faster in the standalone kernels
    // than inside it, and launch overhead is negligible at their size); the others run in
    // one persistent launch, itself a node of that graph
    std::vector<qfx_batch_item> big, small;
    for (int i = 0; i < n_items; ++i) (item_runs_launches(items[i].plan) ? big : small).push_back(items[i]);
    if (!big.empty())
      return prepare_graph(big.data(), (int32_t)big.size(), small, tabmap, workspace, ws_bytes, out, stream);
    return prepare_persistent(items, n_items, tabmap, workspace, ws_bytes, out, stream);
  } catch (const std::exception& ex) {
    return fail(QFX_EINVAL, std::string("qfx_batch_prepare: ") + ex.what());
  }
}

extern "C" qfx_status qfx_batch_run(const qfx_batch* b, void* stream) {
  if (!b) return fail(QFX_EINVAL, "qfx_batch_run: NULL batch");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->exec) {   // graph executor
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_run: capture status");
    if (cs == cudaStreamCaptureStatusActive) {
      // inside a caller's capture: the batch graph becomes a child node of the captured graph
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* edges = nullptr;
      size_t nd = 0;
      cudaGraphNode_t node = nullptr;
      e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &edges, &nd);
      if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&node, cg, deps, nd, b->graph);
      if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_run: adding the batch graph to a capture");
    } else {
      e = cudaGraphLaunch(b->exec, st);
      if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_run: graph launch");
    }
    count_launch((int)b->graph_kernels);
    return QFX_OK;
  }
  cudaError_t e = cudaMemsetAsync(b->control, 0, b->control_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->args.hdrs, 0, b->hdrs_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_run: clearing counters");
  batch_kernel<<<b->grid, kT, b->smem, st>>>(b->args);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "qfx_batch_run: launch");
  return QFX_OK;
}

extern "C" qfx_status qfx_batch_info(const qfx_batch* b, int64_t* n_work, int64_t* n_tasks, int64_t* slots) {
  if (!b) return fail(QFX_EINVAL, "qfx_batch_info: NULL batch");
  if (n_work) *n_work = b->n_work;
  if (n_tasks) *n_tasks = b->args.n_tasks;
  if (slots) *slots = b->slots;
  return QFX_OK;
}

extern "C" void qfx_batch_destroy(qfx_batch* b) { delete b; }

// Test hook: one dependency of the schedule becomes unreachable (its count is raised
// above the tasks that feed it) and every dependency wait is limited to wait_ns, so the
// next qfx_batch_run gives up after wait_ns and qfx_sync reports QFX_ETIMEOUT.
extern "C" qfx_status qfx_debug_batch_stall(qfx_batch* b, int64_t wait_ns) {
  if (!b) return fail(QFX_EINVAL, "qfx_debug_batch_stall: NULL batch");
  if (b->exec) return fail(QFX_EUNSUPPORTED, "qfx_debug_batch_stall: graph batches have no device queue");
  if (wait_ns < 1000 || wait_ns > 5000000000ll)
    return fail(QFX_EINVAL, "qfx_debug_batch_stall: wait_ns must be in [1e3, 5e9]");
  const SegDev* dsegs = b->args.segs;
  for (int32_t i = 0; i < b->args.n_segs; ++i) {
    SegDev sg;
    cudaError_t e = cudaMemcpy(&sg, dsegs + i, sizeof(sg), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_debug_batch_stall");
    if (sg.dep[0] < 0) continue;
    SegDev feed;
    e = cudaMemcpy(&feed, dsegs + sg.dep[0], sizeof(feed), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_debug_batch_stall");
    sg.need[0] = feed.tiles + 1;
    e = cudaMemcpy(const_cast<SegDev*>(dsegs + i), &sg, sizeof(sg), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_debug_batch_stall");
    b->args.wait_ns = (unsigned long long)wait_ns;
    return QFX_OK;
  }
  return fail(QFX_EINVAL, "qfx_debug_batch_stall: the schedule has no dependency");
}
