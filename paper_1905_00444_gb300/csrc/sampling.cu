// Frugal rejection sampling over fast-sampling batches (Sec. III.B).
//
// A batch is the 2^k amplitudes of the bitstrings x1 u x2 that share one x1 (k open
// sites).  Its candidates are examined in the order x2 = t XOR mask, t = 0, 1, ...; the
// candidate at scan position t is accepted when u_t < 2^n |amp|^2 / M.  The first
// accepted candidate is the batch's sample.  Sampling from amplitudes summed over a
// fraction f of the slices is noisy sampling at fidelity about f (Sec. III.C); the caller
// then passes M * f.
//
// One block per batch scans 256 candidates per pass and stops at the first pass with an
// acceptance.  The acceptance is evaluated with explicit round-to-nearest operations
// (p = re*re + im*im, then p * (2^n / M), no fused multiply-add), so the decision is the
// one an FP64 evaluation in that order makes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int kST = 256;

struct OpenSites {
  int16_t q[kMaxOpen];
};

__global__ void __launch_bounds__(kST) frugal_select_kernel(
    const double* __restrict__ amps, const double* __restrict__ u, const uint64_t* __restrict__ scan_mask,
    const uint64_t* __restrict__ x1, int x1_words, int n_open, OpenSites os, double scale,
    int64_t* __restrict__ x2_out, uint64_t* __restrict__ bits_out) {
  __shared__ unsigned long long first;
  const int64_t b = blockIdx.x;
  const int64_t per = int64_t(1) << n_open;
  const uint64_t m = scan_mask[b] & (uint64_t)(per - 1);
  if (threadIdx.x == 0) first = (unsigned long long)per;
  __syncthreads();
  const double* row = amps + 2 * b * per;
  const double* ub = u + b * per;
  for (int64_t t0 = 0; t0 < per; t0 += kST) {
    const int64_t t = t0 + threadIdx.x;
    bool acc = false;
    if (t < per) {
      const int64_t x2 = (int64_t)((uint64_t)t ^ m);
      const double2 a = *reinterpret_cast<const double2*>(row + 2 * x2);
      const double p = __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
      acc = ub[t] < __dmul_rn(p, scale);
    }
    if (__syncthreads_or(acc)) {   // block-uniform
      if (acc) atomicMin(&first, (unsigned long long)t);
      __syncthreads();
      break;
    }
  }
  if (threadIdx.x == 0) {
    const int64_t t = (int64_t)first;
    const int64_t x2 = t < per ? (int64_t)((uint64_t)t ^ m) : -1;
    x2_out[b] = x2;
    if (bits_out) {
      // x1 with each open site's bit replaced by the sample's (x1 unchanged without one)
      for (int wd = 0; wd < x1_words; ++wd) {
        uint64_t bits = x1[b * x1_words + wd];
        if (x2 >= 0)
          for (int i = 0; i < n_open; ++i) {
            if ((os.q[i] >> 6) != wd) continue;
            const uint64_t bit = 1ull << (os.q[i] & 63);
            bits = ((x2 >> i) & 1) ? (bits | bit) : (bits & ~bit);
          }
        bits_out[b * x1_words + wd] = bits;
      }
    }
  }
}

}  // namespace
}  // namespace qfx

using namespace qfx;

extern "C" qfx_status qfx_frugal_select(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                        const double* amps, const double* u,
                                        const uint64_t* scan_mask, double M, int64_t* x2_out,
                                        uint64_t* bits_out, void* stream) {
  if (!p) return fail(QFX_EINVAL, "qfx_frugal_select: NULL plan");
  if (n_batch < 0) return fail(QFX_EINVAL, "qfx_frugal_select: negative n_batch");
  if (!(M > 0.0) || !std::isfinite(M)) return fail(QFX_EINVAL, "qfx_frugal_select: M must be finite and > 0");
  if (n_batch == 0) return QFX_OK;
  if (!x1 || !amps || !u || !scan_mask || !x2_out) return fail(QFX_EINVAL, "qfx_frugal_select: NULL argument");
  if (n_batch > 0x7fffffff) return fail(QFX_EINVAL, "qfx_frugal_select: n_batch above 2^31 - 1");
  if (reinterpret_cast<uintptr_t>(amps) & 15) return fail(QFX_EINVAL, "qfx_frugal_select: amps not 16-byte aligned");
  const int n_open = (int)p->open_sites.size();
  if (n_open > kMaxOpen) return fail(QFX_EINVAL, "qfx_frugal_select: more than 24 open sites");
  OpenSites os{};
  for (int i = 0; i < n_open; ++i) os.q[i] = (int16_t)p->open_sites[i];
  const double scale = std::ldexp(1.0, p->rows * p->cols) / M;
  int slot;
  profile_begin(stream, &slot);
  frugal_select_kernel<<<(unsigned)n_batch, kST, 0, (cudaStream_t)stream>>>(
      amps, u, scan_mask, x1, p->x1_words, n_open, os, scale, x2_out, bits_out);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  profile_end(stream, slot, -1, 0, 5, 0.0, (double)n_batch * (24.0 * (double)(int64_t(1) << n_open) + 24.0));
  if (e != cudaSuccess) return cuda_fail(e, "qfx_frugal_select");
  return QFX_OK;
}
