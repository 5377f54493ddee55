// Per-element time fold of one site tensor (Sec. III, Fig. 3), shared by fold.cu and the
// batch scheduler.  See fold.cu for the method.
#pragma once
#include <cuda_runtime.h>

#include "qfx_internal.h"

namespace qfx {
namespace foldk {

// Float-float ("double-single") arithmetic: a real value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits, on the FP32
// pipes (this GPU runs FP64 at 1/64 of the FP32 rate).  Built from two error-free
// transformations: Knuth's TwoSum (s + e = a + b exactly) and the product's exact error
// by a fused multiply-add (a*b - fl(a*b), Dekker's TwoProduct with FMA); the sum and
// product below follow Dekker's double-length algorithms (1971).  Every step is an
// explicit round-to-nearest intrinsic, which the compiler never contracts or reorders, so
// every caller rounds exactly alike: the group fold relies on it to reproduce the
// per-element fold bit for bit.
struct ff {
  float hi, lo;
};
struct cff {
  ff re, im;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // needs |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);   // exact: a.hi * b.hi = p + e
  return fast_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ cff cmul(cff a, cff b) {
  return {ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))),
          ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ __forceinline__ cff cadd(cff a, cff b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
// complex entry j (re at 2j, im at 2j + 1 of the FP64 layout) of a float-float matrix
__device__ __forceinline__ cff centry(const float* __restrict__ m, int j) {
  return {{m[2 * j], m[2 * j + 1]}, {m[2 * j + 2], m[2 * j + 3]}};
}
__device__ __forceinline__ float ff_round(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ cff cff_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cff cff_one() { return {{1.f, 0.f}, {0.f, 0.f}}; }

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
// the 2x2 block B_k on q1 of a general one.  `matsf` holds each matrix's 8 FP64 entries
// (re, im of the 2x2 complex matrix, row-major) as 16 floats, a (hi, lo) pair per entry.
__device__ __forceinline__ void apply_event(const FoldEvent& ev, const float* __restrict__ matsf, int k,
                                            cff& v0, cff& v1) {
  const float* m = matsf + 16 * (int64_t)ev.mat;
  if (ev.kind == EV_GATE || ev.kind == EV_BLOCK) {
    const float* b = ev.kind == EV_GATE ? m : m + 16 * k;
    const cff n0 = cadd(cmul(centry(b, 0), v0), cmul(centry(b, 2), v1));
    const cff n1 = cadd(cmul(centry(b, 4), v0), cmul(centry(b, 6), v1));
    v0 = n0;
    v1 = n1;
  } else if (ev.kind == EV_PROJ) {
    if (k) v0 = cff_zero();
    else   v1 = cff_zero();
  } else if (ev.kind == EV_DIAG) {
    v0 = cmul(v0, centry(m, 4 * k + 0));
    v1 = cmul(v1, centry(m, 4 * k + 2));
  } else {   // EV_ELEM: |o0><i0|
    const cff src = (k & 1) ? v1 : v0;
    v0 = (k >> 1) ? cff_zero() : src;
    v1 = (k >> 1) ? src : cff_zero();
  }
}

// Element i of site `st` for slice `sid`: float-float evolution of the site's 2-vector
// through its time line from |0>, rounded once to complex64.
__device__ __forceinline__ float2 fold_element(const FoldSite& st, const FoldEvent* __restrict__ events,
                                               const float* __restrict__ matsf,
                                               const CutDev* __restrict__ cuts, int n_cuts,
                                               const uint64_t* __restrict__ x1w, int64_t sid,
                                               int64_t i) {
  const FoldCoord fc = fold_coord(st, cuts, n_cuts, x1w, sid, i);
  cff v0 = cff_one(), v1 = cff_zero();
  for (int e = st.ev_begin; e < st.ev_end; ++e) {
    const FoldEvent ev = events[e];
    apply_event(ev, matsf, event_key(ev, fc), v0, v1);
  }
  const cff res = fc.xv ? v1 : v0;
  return make_float2(ff_round(res.re), ff_round(res.im));
}

}  // namespace foldk
}  // namespace qfx
