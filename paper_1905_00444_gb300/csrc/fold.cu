// Site-tensor builder (time-first folding), per-site power-of-two normalisation, and the
// FP64 sum of slice contributions.
//
// Fold (Sec. III, Fig. 3): for grid site q, the gates on its time line are applied to
// |0> in order; a diagonal two-qubit gate D between q0 and q1 is split as
// D(b0, b1) = sum_k delta(b0, k) D(k, b1), so q0 applies the projector |k><k| and q1
// applies diag(D(k,0), D(k,1)), with k one bit (leg) of the bond between them.  The
// tensor element T[up][left][x][right][down] is <x| ... |0> for the leg bits that its
// bond values carry.  One thread computes one element in FP64 and rounds it once to
// complex64.
//
// Normalisation (Sec. III.E: inputs normalised, outputs renormalised, to keep FP32
// away from underflow): each site is scaled by 2^-e with e chosen so that its largest
// |re| or |im| lies in [1/2, 1); the exponents are summed per work item and undone in
// FP64 when the slice contributions are added (Sec. III.A: sum over paths).
#include <cuda_runtime.h>

#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

__global__ void __launch_bounds__(kThreads) fold_kernel(
    const FoldSite* __restrict__ sites, const FoldEvent* __restrict__ events,
    const double* __restrict__ mats, const CutDev* __restrict__ cuts, int n_cuts,
    const uint64_t* __restrict__ x1, int64_t n_batch, int64_t slice_begin, int64_t item0,
    char* hdr, uint64_t hdr_stride, char* items, uint64_t item_bytes, uint64_t sites_off,
    int n_sites) {
  const FoldSite st = sites[blockIdx.y];
  const int g = blockIdx.z;
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool active = i < st.size;
  float mx = 0.f;
  if (active) {
    const int64_t item = item0 + g;
    const int64_t b = item % n_batch;
    const int64_t sid = slice_begin + item / n_batch;
    int64_t off[4] = {0, 0, 0, 0};
    for (int c = 0; c < n_cuts; ++c) {
      const CutDev cd = cuts[c];
      const int64_t digit = (sid / cd.suffix) % cd.radix;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (st.edge[s] == cd.edge) off[s] = digit * cd.size;
    }
    int64_t r = i;
    const int64_t vd = r % st.dim[4]; r /= st.dim[4];
    const int64_t vr = r % st.dim[3]; r /= st.dim[3];
    const int64_t vx = r % st.dim[2]; r /= st.dim[2];
    const int64_t vl = r % st.dim[1]; r /= st.dim[1];
    const int64_t vu = r;
    const uint64_t val0 = (uint64_t)(vu + off[0]), val1 = (uint64_t)(vl + off[1]);
    const uint64_t val2 = (uint64_t)(vr + off[2]), val3 = (uint64_t)(vd + off[3]);
    const int xv = st.x_open ? (int)vx : (int)((x1[b] >> st.qubit) & 1ull);
    double2 v0 = make_double2(1.0, 0.0), v1 = make_double2(0.0, 0.0);
    for (int e = st.ev_begin; e < st.ev_end; ++e) {
      const FoldEvent ev = events[e];
      const double* m = mats + 8 * (int64_t)ev.mat;
      if (ev.kind == EV_GATE) {
        const double2 g00 = make_double2(m[0], m[1]), g01 = make_double2(m[2], m[3]);
        const double2 g10 = make_double2(m[4], m[5]), g11 = make_double2(m[6], m[7]);
        const double2 n0 = cadd(cmul(g00, v0), cmul(g01, v1));
        const double2 n1 = cadd(cmul(g10, v0), cmul(g11, v1));
        v0 = n0;
        v1 = n1;
      } else {
        const uint64_t bv = ev.slot == 0 ? val0 : ev.slot == 1 ? val1 : ev.slot == 2 ? val2 : val3;
        const int k = (int)((bv >> ev.bit) & 1ull);
        if (ev.kind == EV_PROJ) {
          if (k) v0 = make_double2(0.0, 0.0);
          else   v1 = make_double2(0.0, 0.0);
        } else {
          v0 = cmul(v0, make_double2(m[4 * k + 0], m[4 * k + 1]));
          v1 = cmul(v1, make_double2(m[4 * k + 2], m[4 * k + 3]));
        }
      }
    }
    const double2 res = xv ? v1 : v0;
    const float2 out = make_float2((float)res.x, (float)res.y);
    float2* T = reinterpret_cast<float2*>(items + (uint64_t)g * item_bytes + sites_off) + st.offset;
    T[i] = out;
    mx = fmaxf(fabsf(out.x), fabsf(out.y));
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
                const uint64_t* x1, int64_t n_batch, int64_t slice_begin, int64_t item0,
                int items, char* hdr, uint64_t hdr_stride, char* itemsp, uint64_t item_bytes,
                uint64_t sites_off, void* stream) {
  dim3 grid((unsigned)((max_site_size + kThreads - 1) / kThreads), n_sites, items);
  fold_kernel<<<grid, kThreads, 0, (cudaStream_t)stream>>>(
      t.sites, t.events, t.mats, t.cuts, n_cuts, x1, n_batch, slice_begin, item0, hdr,
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
