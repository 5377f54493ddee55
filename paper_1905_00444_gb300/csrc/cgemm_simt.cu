// One contraction step as a complex FP32 GEMM on the FMA pipes (the plain path): one
// launch per step, one CTA per output tile (tile body in cgemm_tile.cuh).
#include <cuda_runtime.h>

#include <cstdio>

#include "cgemm_tile.cuh"
#include "qfx_internal.h"

namespace qfx {
namespace {
using namespace simt;

template <int BM, int BJ, int TM, int TJ, bool KMODE, int STAGES, int NTH>
__global__ void __launch_bounds__(NTH) cgemm_step_kernel(const StepArgs a) {
  extern __shared__ float4 smem_raw[];
  cgemm_tile<BM, BJ, TM, TJ, KMODE, STAGES, NTH>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Shared-memory opt-in of one tile kernel, once per device (also called ahead of a graph
// capture, which must not be the first launch to set it).
template <int BM, int BJ, int TM, int TJ, bool KMODE, int STAGES, int NTH = 256>
int ensure_attr() {
  using C_ = Cfg<BM, BJ, TM, TJ, KMODE, STAGES, NTH>;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_step_kernel<BM, BJ, TM, TJ, KMODE, STAGES, NTH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_::SMEM);
    if (e != cudaSuccess) return (int)e;
    attr_done[dev] = 1;
  }
  return 0;
}

template <int BM, int BJ, int TM, int TJ, bool KMODE, int STAGES, int NTH = 256>
int launch_cfg(const StepArgs& a, int batch, cudaStream_t stream) {
  using C_ = Cfg<BM, BJ, TM, TJ, KMODE, STAGES, NTH>;
  auto kern = cgemm_step_kernel<BM, BJ, TM, TJ, KMODE, STAGES, NTH>;
  if (int e = ensure_attr<BM, BJ, TM, TJ, KMODE, STAGES, NTH>()) return e;
  const int64_t NT = (a.N + BM - 1) / BM;
  const int64_t JT = (a.J + BJ - 1) / BJ;
  const int64_t blocks = NT * JT;
  if (blocks > 0x7fffffffLL || batch > 65535) return (int)cudaErrorInvalidConfiguration;
  kern<<<dim3((unsigned)blocks, batch), NTH, C_::SMEM, stream>>>(a);
  count_launch();
  return (int)cudaGetLastError();
}

// Split-K sum of a chunked contraction.  A block covers kRedE consecutive outputs with
// kRedL lanes each: lane l of an output adds chunks l, l + kRedL, ... in FP64 (a warp reads
// kRedE-long runs of each chunk's row), then lane 0 adds the lanes' sums in lane order and
// rounds once to FP32.
constexpr int kRedE = 32, kRedL = 8;
__global__ void __launch_bounds__(kRedE * kRedL) reduce_parts_kernel(const float2* __restrict__ part,
                                                                     int64_t part_stride, int64_t parts,
                                                                     int64_t out, float2* __restrict__ C,
                                                                     int64_t c_stride) {
  __shared__ double2 lanes[kRedL][kRedE];
  const int el = threadIdx.x % kRedE, lane = threadIdx.x / kRedE;
  const int64_t e = (int64_t)blockIdx.x * kRedE + el;
  const float2* pp = part + (int64_t)blockIdx.y * part_stride;
  double re = 0.0, im = 0.0;
  if (e < out) {
#pragma unroll 4
    for (int64_t c = lane; c < parts; c += kRedL) {
      const float2 v = pp[c * out + e];
      re += (double)v.x;
      im += (double)v.y;
    }
  }
  lanes[lane][el] = make_double2(re, im);
  __syncthreads();
  if (lane == 0 && e < out) {
    for (int l = 1; l < kRedL; ++l) {
      re += lanes[l][el].x;
      im += lanes[l][el].y;
    }
    C[(int64_t)blockIdx.y * c_stride + e] = make_float2((float)re, (float)im);
  }
}

}  // namespace

int launch_reduce_parts(const void* part, int64_t part_stride, int64_t parts, int64_t out, void* C,
                        int64_t c_stride, int batch, void* stream) {
  if (parts < 1 || out < 1 || batch < 1 || batch > 65535) return (int)cudaErrorInvalidValue;
  const int64_t blocks = (out + kRedE - 1) / kRedE;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
  reduce_parts_kernel<<<dim3((unsigned)blocks, (unsigned)batch), kRedE * kRedL, 0, (cudaStream_t)stream>>>(
      (const float2*)part, part_stride, parts, out, (float2*)C, c_stride);
  count_launch();
  return (int)cudaGetLastError();
}

int simt_prepare_attributes() {
#define QFX_ATTR(V, BM, BJ, TM, TJ, KM, ST) \
  if (int e = ensure_attr<BM, BJ, TM, TJ, KM, ST>()) return e;
  QFX_SIMT_VARIANTS(QFX_ATTR)
#undef QFX_ATTR
#define QFX_ATTR(V, BM, BJ, TM, TJ, KM, ST, NT) \
  if (int e = ensure_attr<BM, BJ, TM, TJ, KM, ST, NT>()) return e;
  QFX_SIMT_FILL_VARIANTS(QFX_ATTR)
#undef QFX_ATTR
  return 0;
}

// Tile variants (QFX_SIMT_VARIANTS): 0..4 stream B along s (JMODE), 5..9 load B along k.
int pick_variant(int64_t N, int64_t Sd) {
  int base = N >= 128 ? 0 : N >= 64 ? 1 : N >= 32 ? 2 : N >= 16 ? 3 : 4;
  return base + ((Sd % 2) ? 5 : 0);
}

int num_sms() {
  static int n[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64) dev = 63;
  if (!n[dev]) cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
  return n[dev] > 0 ? n[dev] : 1;
}

// Variants 0..9 keep their tile when its grid gives at least two CTAs per SM; otherwise the
// fill variant of the same row range (QFX_SIMT_FILL_VARIANTS) when it gives more CTAs.
// Both sum every output's k terms in the same order, so the choice never changes a result.
int fill_variant(int variant, int64_t N, int64_t J, int batch) {
  static const int bm[10] = {128, 64, 32, 16, 8, 128, 64, 32, 16, 8};
  static const int bj[10] = {128, 256, 512, 512, 512, 128, 256, 512, 512, 512};
  static const int fill[10] = {20, 20, 21, 22, 23, 25, 25, 26, 27, 28};
  static const int fbm[10] = {64, 64, 32, 16, 8, 64, 64, 32, 16, 8};
  static const int fbj[10] = {64, 64, 128, 256, 256, 64, 64, 128, 256, 256};
  if (variant < 0 || variant > 9 || batch < 1) return variant;
  const int64_t blocks = ((N + bm[variant] - 1) / bm[variant]) * ((J + bj[variant] - 1) / bj[variant]) * batch;
  if (blocks >= 2 * (int64_t)num_sms()) return variant;
  const int64_t fb = ((N + fbm[variant] - 1) / fbm[variant]) * ((J + fbj[variant] - 1) / fbj[variant]) * batch;
  return fb > blocks ? fill[variant] : variant;
}

bool simt_variant_valid(int variant, int64_t Sd) {
  const bool jmode = (variant >= 0 && variant < 5) || (variant >= 20 && variant < 24);
  const bool kmode = (variant >= 5 && variant < 10) || (variant >= 25 && variant < 29);
  return (jmode && Sd % 2 == 0) || kmode;
}

int launch_step(const void* S, int64_t s_stride, const void* B, int64_t b_stride, void* C,
                int64_t c_stride, int64_t P, int64_t K, int64_t N, int64_t NL, int64_t Sd,
                int batch, int variant, int precision, void* stream, int beta) {
  (void)precision;
  StepArgs a{(const float2*)S, s_stride, (const float2*)B, b_stride, (float2*)C, c_stride,
             P, K, N, NL, Sd, P * Sd, beta};
  if (variant < 0) variant = pick_variant(N, Sd);
  if (!simt_variant_valid(variant, Sd)) return (int)cudaErrorInvalidValue;  // JMODE needs even Sd
  cudaStream_t st = (cudaStream_t)stream;
  switch (variant) {
#define QFX_CASE(V, BM, BJ, TM, TJ, KM, ST) \
  case V: return launch_cfg<BM, BJ, TM, TJ, KM, ST>(a, batch, st);
    QFX_SIMT_VARIANTS(QFX_CASE)
#undef QFX_CASE
#define QFX_CASE(V, BM, BJ, TM, TJ, KM, ST, NT) \
  case V: return launch_cfg<BM, BJ, TM, TJ, KM, ST, NT>(a, batch, st);
    QFX_SIMT_FILL_VARIANTS(QFX_CASE)
#undef QFX_CASE
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace qfx
