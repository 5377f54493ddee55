// Site-tensor builder (time-first folding), per-site power-of-two normalisation, and the
// FP64 sum of slice contributions.
//
// Fold (Sec. III, Fig. 3): for grid site q, the gates on its time line are applied to
// |0> in order; a diagonal two-qubit gate D between q0 and q1 is split as
// D(b0, b1) = sum_k delta(b0, k) D(k, b1), so q0 applies the projector |k><k| and q1
// applies diag(D(k,0), D(k,1)), with k one bit (leg) of the bond between them.  The
// tensor element T[up][left][x][right][down] is <x| ... |0> for the leg bits that its
// bond values carry.  Each element is evolved in float-float arithmetic (FP32 pairs,
// about 48 significant bits; see fold_element.cuh) and rounded once to complex64.  A
// thread takes kGroup consecutive elements: they differ only in the low bits of the
// innermost bond (its latest gates), so up to the first event that reads one of those bits
// they share one 2-vector, computed once with the same operations as each element's own
// fold (the results are those of foldk::fold_element bit for bit); from there on each
// element has its own.
//
// Normalisation (Sec. III.E: inputs normalised, outputs renormalised, to keep FP32
// away from underflow): each site is scaled by 2^-e with e chosen so that its largest
// |re| or |im| lies in [1/2, 1); the exponents are summed per work item and undone in
// FP64 when the slice contributions are added (Sec. III.A: sum over paths).
#include <cuda_runtime.h>

#include "fold_element.cuh"
#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 4;   // consecutive elements per thread

template <int G>
__device__ __forceinline__ void fold_group(const FoldSite& st, const FoldEvent* __restrict__ events,
                                           const float* __restrict__ matsf, const CutDev* __restrict__ cuts,
                                           int n_cuts, const uint64_t* __restrict__ x1w, int64_t sid,
                                           int64_t i0, float2 out[G]) {
  foldk::FoldCoord fc[G];
#pragma unroll
  for (int q = 0; q < G; ++q) fc[q] = foldk::fold_coord(st, cuts, n_cuts, x1w, sid, i0 + q);
  foldk::cff v0[G], v1[G];
  v0[0] = foldk::cff_one();
  v1[0] = foldk::cff_zero();
  bool split = false;
  for (int e = st.ev_begin; e < st.ev_end; ++e) {
    const FoldEvent ev = events[e];
    int k[G];
#pragma unroll
    for (int q = 0; q < G; ++q) k[q] = foldk::event_key(ev, fc[q]);
    if (!split) {
      bool same = true;
#pragma unroll
      for (int q = 1; q < G; ++q) same = same && k[q] == k[0];
      if (same) {
        foldk::apply_event(ev, matsf, k[0], v0[0], v1[0]);
        continue;
      }
#pragma unroll
      for (int q = 1; q < G; ++q) { v0[q] = v0[0]; v1[q] = v1[0]; }
      split = true;
    }
#pragma unroll
    for (int q = 0; q < G; ++q) foldk::apply_event(ev, matsf, k[q], v0[q], v1[q]);
  }
  if (!split) {
#pragma unroll
    for (int q = 1; q < G; ++q) { v0[q] = v0[0]; v1[q] = v1[0]; }
  }
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const foldk::cff res = fc[q].xv ? v1[q] : v0[q];
    out[q] = make_float2(foldk::ff_round(res.re), foldk::ff_round(res.im));
  }
}

__global__ void __launch_bounds__(kThreads) fold_kernel(
    const FoldSite* __restrict__ sites, const FoldEvent* __restrict__ events,
    const float* __restrict__ matsf, const CutDev* __restrict__ cuts, int n_cuts,
    const uint64_t* __restrict__ x1, int x1_words, int64_t n_batch, int64_t slice_begin,
    int64_t item0, char* hdr, uint64_t hdr_stride, char* items, uint64_t item_bytes,
    uint64_t sites_off, int n_sites) {
  const FoldSite st = sites[blockIdx.y];
  const int g = blockIdx.z;
  const int64_t i0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * kGroup;
  float mx = 0.f;
  if (i0 < st.size) {
    const int64_t item = item0 + g;
    const int64_t b = item % n_batch;
    const int64_t sid = slice_begin + item / n_batch;
    float2 out[kGroup];
    fold_group<kGroup>(st, events, matsf, cuts, n_cuts, x1 + b * x1_words, sid, i0, out);
    float2* T = reinterpret_cast<float2*>(items + (uint64_t)g * item_bytes + sites_off) + st.offset;
#pragma unroll
    for (int q = 0; q < kGroup; ++q)
      if (i0 + q < st.size) {
        T[i0 + q] = out[q];
        mx = fmaxf(mx, fmaxf(fabsf(out[q].x), fabsf(out[q].y)));
      }
  }
  // non-negative floats order like their bit patterns
  const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  if ((threadIdx.x & 31) == 0 && bits) {
    unsigned* maxabs = reinterpret_cast<unsigned*>(hdr + (uint64_t)g * hdr_stride);
    atomicMax(maxabs + blockIdx.y, bits);
  }
}

__global__ void __launch_bounds__(kThreads) scale_kernel(
    const FoldSite* __restrict__ sites, char* hdr, uint64_t hdr_stride, char* items,
    uint64_t item_bytes, uint64_t sites_off, int n_sites) {
  const FoldSite st = sites[blockIdx.y];
  const int g = blockIdx.z;
  const unsigned* maxabs = reinterpret_cast<const unsigned*>(hdr + (uint64_t)g * hdr_stride);
  const float m = __uint_as_float(maxabs[blockIdx.y]);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int* exps = reinterpret_cast<int*>(hdr + (uint64_t)g * hdr_stride) + n_sites;
    exps[blockIdx.y] = e;
  }
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= st.size || e == 0) return;
  const float sc = ldexpf(1.0f, -e);
  float2* T = reinterpret_cast<float2*>(items + (uint64_t)g * item_bytes + sites_off) + st.offset;
  float2 v = T[i];
  v.x *= sc;
  v.y *= sc;
  T[i] = v;
}

__global__ void __launch_bounds__(kThreads) accumulate_kernel(
    const int32_t* __restrict__ open_perm, int n_open, int n_sites, int64_t n_batch,
    int64_t item0, int items, const char* hdr, uint64_t hdr_stride, const char* itemsp,
    uint64_t item_bytes, uint64_t final_off, double* out) {
  const int64_t per = int64_t(1) << n_open;
  const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= n_batch * per) return;
  const int64_t b = t / per, o = t % per;
  int64_t f = 0;
  for (int i = 0; i < n_open; ++i) f |= ((o >> i) & 1) << open_perm[i];
  // items of this chunk with batch index b, in increasing slice order
  int64_t first = item0 + ((b - item0 % n_batch) % n_batch + n_batch) % n_batch;
  double re = out[2 * t], im = out[2 * t + 1];
  bool any = false;
  for (int64_t item = first; item < item0 + items; item += n_batch) {
    const int g = (int)(item - item0);
    const int* exps = reinterpret_cast<const int*>(hdr + (uint64_t)g * hdr_stride) + n_sites;
    int E = 0;
    for (int s = 0; s < n_sites; ++s) E += exps[s];
    const float2 c = reinterpret_cast<const float2*>(itemsp + (uint64_t)g * item_bytes + final_off)[f];
    re += ldexp((double)c.x, E);
    im += ldexp((double)c.y, E);
    any = true;
  }
  if (any) {
    out[2 * t] = re;
    out[2 * t + 1] = im;
  }
}

}  // namespace

int launch_fold(const DeviceTables& t, int n_sites, int64_t max_site_size, int n_cuts,
                const uint64_t* x1, int x1_words, int64_t n_batch, int64_t slice_begin,
                int64_t item0, int items, char* hdr, uint64_t hdr_stride, char* itemsp,
                uint64_t item_bytes, uint64_t sites_off, void* stream) {
  const int64_t per_block = (int64_t)kThreads * kGroup;
  dim3 grid((unsigned)((max_site_size + per_block - 1) / per_block), n_sites, items);
  fold_kernel<<<grid, kThreads, 0, (cudaStream_t)stream>>>(
      t.sites, t.events, t.matsf, t.cuts, n_cuts, x1, x1_words, n_batch, slice_begin, item0, hdr,
      hdr_stride, itemsp, item_bytes, sites_off, n_sites);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_scale(const DeviceTables& t, int n_sites, int64_t max_site_size, int items,
                 char* hdr, uint64_t hdr_stride, char* itemsp, uint64_t item_bytes,
                 uint64_t sites_off, void* stream) {
  dim3 grid((unsigned)((max_site_size + kThreads - 1) / kThreads), n_sites, items);
  scale_kernel<<<grid, kThreads, 0, (cudaStream_t)stream>>>(t.sites, hdr, hdr_stride, itemsp,
                                                             item_bytes, sites_off, n_sites);
  count_launch();
  return (int)cudaGetLastError();
}

int launch_accumulate(const DeviceTables& t, int n_sites, int n_open, int64_t n_batch,
                      int64_t item0, int items, const char* hdr, uint64_t hdr_stride,
                      const char* itemsp, uint64_t item_bytes, uint64_t final_off, double* out,
                      void* stream) {
  const int64_t total = n_batch << n_open;
  const unsigned blocks = (unsigned)((total + kThreads - 1) / kThreads);
  accumulate_kernel<<<blocks, kThreads, 0, (cudaStream_t)stream>>>(
      t.open_perm, n_open, n_sites, n_batch, item0, items, hdr, hdr_stride, itemsp, item_bytes,
      final_off, out);
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace qfx
