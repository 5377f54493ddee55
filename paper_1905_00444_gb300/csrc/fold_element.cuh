// Per-element time fold of one site tensor (Sec. III, Fig. 3), shared by fold.cu and the
// batch scheduler.  See fold.cu for the method.
#pragma once
#include <cuda_runtime.h>

#include "qfx_internal.h"

namespace qfx {
namespace foldk {

// Complex FP64 products with the rounding steps written out (one product, one fused
// multiply-add per part), so that every caller rounds exactly alike whatever the compiler
// would contract in its context: the group fold below relies on it to reproduce the
// per-element fold bit for bit.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}

// Bond values (up, left, right, down, each plus its cut offset for slice `sid`) and the x
// value of element i of site `st`; the output bitstring x1w is given as words (qubit q is
// bit q % 64 of word q / 64).
struct FoldCoord {
  uint64_t val[4];
  int xv;
};
__device__ __forceinline__ FoldCoord fold_coord(const FoldSite& st, const CutDev* __restrict__ cuts, int n_cuts,
                                                const uint64_t* __restrict__ x1w, int64_t sid, int64_t i) {
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
  FoldCoord fc;
  fc.val[0] = (uint64_t)(vu + off[0]);
  fc.val[1] = (uint64_t)(vl + off[1]);
  fc.val[2] = (uint64_t)(vr + off[2]);
  fc.val[3] = (uint64_t)(vd + off[3]);
  fc.xv = st.x_open ? (int)vx : (int)((x1w[st.qubit >> 6] >> (st.qubit & 63)) & 1ull);
  return fc;
}

// The bond bits an event reads for an element (0 for a one-qubit gate): one bit for a
// diagonal two-qubit gate, two (k = 2*o0 + i0) for a general one.
__device__ __forceinline__ int event_key(const FoldEvent& ev, const FoldCoord& fc) {
  if (ev.kind == EV_GATE) return 0;
  const uint64_t bv = ev.slot == 0 ? fc.val[0] : ev.slot == 1 ? fc.val[1] : ev.slot == 2 ? fc.val[2] : fc.val[3];
  const uint64_t mask = (ev.kind == EV_PROJ || ev.kind == EV_DIAG) ? 1ull : 3ull;
  return (int)((bv >> ev.bit) & mask);
}

// One event on the site's 2-vector (v0, v1), for bond bits k: a one-qubit gate; the
// projector on q0 or the diagonal on q1 of a diagonal two-qubit gate; |o0><i0| on q0 or
// the 2x2 block B_k on q1 of a general one.
__device__ __forceinline__ void apply_event(const FoldEvent& ev, const double* __restrict__ mats, int k,
                                            double2& v0, double2& v1) {
  const double* m = mats + 8 * (int64_t)ev.mat;
  if (ev.kind == EV_GATE || ev.kind == EV_BLOCK) {
    const double* b = ev.kind == EV_GATE ? m : m + 8 * k;
    const double2 n0 = cadd(cmul(make_double2(b[0], b[1]), v0), cmul(make_double2(b[2], b[3]), v1));
    const double2 n1 = cadd(cmul(make_double2(b[4], b[5]), v0), cmul(make_double2(b[6], b[7]), v1));
    v0 = n0;
    v1 = n1;
  } else if (ev.kind == EV_PROJ) {
    if (k) v0 = make_double2(0.0, 0.0);
    else   v1 = make_double2(0.0, 0.0);
  } else if (ev.kind == EV_DIAG) {
    v0 = cmul(v0, make_double2(m[4 * k + 0], m[4 * k + 1]));
    v1 = cmul(v1, make_double2(m[4 * k + 2], m[4 * k + 3]));
  } else {   // EV_ELEM: |o0><i0|
    const double2 src = (k & 1) ? v1 : v0;
    v0 = (k >> 1) ? make_double2(0.0, 0.0) : src;
    v1 = (k >> 1) ? src : make_double2(0.0, 0.0);
  }
}

// Element i of site `st` for slice `sid`: FP64 evolution of the site's 2-vector through
// its time line from |0>, rounded once to complex64.
__device__ __forceinline__ float2 fold_element(const FoldSite& st, const FoldEvent* __restrict__ events,
                                               const double* __restrict__ mats,
                                               const CutDev* __restrict__ cuts, int n_cuts,
                                               const uint64_t* __restrict__ x1w, int64_t sid,
                                               int64_t i) {
  const FoldCoord fc = fold_coord(st, cuts, n_cuts, x1w, sid, i);
  double2 v0 = make_double2(1.0, 0.0), v1 = make_double2(0.0, 0.0);
  for (int e = st.ev_begin; e < st.ev_end; ++e) {
    const FoldEvent ev = events[e];
    apply_event(ev, mats, event_key(ev, fc), v0, v1);
  }
  const double2 res = fc.xv ? v1 : v0;
  return make_float2((float)res.x, (float)res.y);
}

}  // namespace foldk
}  // namespace qfx
