// Per-element time fold of one site tensor (Sec. III, Fig. 3), shared by fold.cu and the
// batch scheduler.  See fold.cu for the method.
#pragma once
#include <cuda_runtime.h>

#include "qfx_internal.h"

namespace qfx {
namespace foldk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

// Element i of site `st` for slice `sid` and the output bitstring x1w (its words; qubit q
// is bit q % 64 of word q / 64): FP64 evolution of the
// site's 2-vector through its time line, rounded once to complex64.  A diagonal two-qubit
// gate reads one bit of the bond value (projector on q0, diagonal on q1); a general one
// reads two, k = 2*o0 + i0 (|o0><i0| on q0, the 2x2 block B_k of the gate on q1).
__device__ __forceinline__ float2 fold_element(const FoldSite& st, const FoldEvent* __restrict__ events,
                                               const double* __restrict__ mats,
                                               const CutDev* __restrict__ cuts, int n_cuts,
                                               const uint64_t* __restrict__ x1w, int64_t sid,
                                               int64_t i) {
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
  const int xv = st.x_open ? (int)vx : (int)((x1w[st.qubit >> 6] >> (st.qubit & 63)) & 1ull);
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
      if (ev.kind == EV_PROJ || ev.kind == EV_DIAG) {
        const int k = (int)((bv >> ev.bit) & 1ull);
        if (ev.kind == EV_PROJ) {
          if (k) v0 = make_double2(0.0, 0.0);
          else   v1 = make_double2(0.0, 0.0);
        } else {
          v0 = cmul(v0, make_double2(m[4 * k + 0], m[4 * k + 1]));
          v1 = cmul(v1, make_double2(m[4 * k + 2], m[4 * k + 3]));
        }
      } else {
        const int k = (int)((bv >> ev.bit) & 3ull);   // k = 2*o0 + i0
        if (ev.kind == EV_ELEM) {                      // |o0><i0|
          const double2 src = (k & 1) ? v1 : v0;
          v0 = (k >> 1) ? make_double2(0.0, 0.0) : src;
          v1 = (k >> 1) ? src : make_double2(0.0, 0.0);
        } else {                                       // B_k
          const double* b = m + 8 * k;
          const double2 n0 = cadd(cmul(make_double2(b[0], b[1]), v0), cmul(make_double2(b[2], b[3]), v1));
          const double2 n1 = cadd(cmul(make_double2(b[4], b[5]), v0), cmul(make_double2(b[6], b[7]), v1));
          v0 = n0;
          v1 = n1;
        }
      }
    }
  }
  const double2 res = xv ? v1 : v0;
  return make_float2((float)res.x, (float)res.y);
}

}  // namespace foldk
}  // namespace qfx
