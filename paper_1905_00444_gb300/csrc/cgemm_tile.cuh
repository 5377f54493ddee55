// Tile body of the FP32 SIMT contraction step, shared by the per-step kernels
// (cgemm_simt.cu) and the persistent batch scheduler (batch.cu).
//
//   C[nh][p][nl][s] = sum_k S[k][nh*NL + nl] * B[p][k][s]
//
// is the TTGT contraction of Sec. III.E with the transposes folded into the addressing:
// rows are n (M = N), columns are j = p*Sd + s (J = P*Sd), the reduction is k.  Eq. 1
// counts 8*N*J*K flops; each complex multiply-add is 4 real FMAs (the paper's complex
// FP32 CGEMM, without tensor cores).
//
// Tiling: one CTA computes BM x BJ outputs with NTH threads (256 unless a variant says
// otherwise), each thread TM x TJ; the
// k loop moves BK = 8 slabs of S and B through a STAGES-deep cp.async ring in shared
// memory.  Column fragments are read as 2-complex (16-byte) vectors spaced so that 8
// consecutive lanes cover 128 contiguous bytes (no bank conflicts); row fragments are
// warp broadcasts.  JMODE loads B as 16-byte vectors along s (Sd even); KMODE loads it
// element by element (Sd odd, e.g. the last site of a line where Sd = 1).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace qfx {
namespace simt {

struct StepArgs {
  const float2* S; int64_t s_stride;
  const float2* B; int64_t b_stride;
  float2* C; int64_t c_stride;
  int64_t P, K, N, NL, Sd, J;
  int32_t beta;   // 1: add the product into C (a chunk of a long contraction), 0: write it
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int BK = 8;

template <int BM, int BJ, int TM, int TJ, bool KMODE, int STAGES, int NTH = 256>
struct Cfg {
  static constexpr int TYN = BM / TM, TXN = BJ / TJ;
  static constexpr int LDA = BM + 2, LDB = BJ + 2;
  static constexpr int A_IT = (BK * BM + NTH - 1) / NTH;
  static constexpr int B_IT = KMODE ? (BK * BJ) / NTH : (BK * BJ) / (2 * NTH);
  static constexpr size_t SMEM = (size_t)STAGES * BK * (LDA + LDB) * sizeof(float2);
  static_assert(TYN * TXN == NTH, "one thread per TM x TJ outputs");
  static_assert(TM % 2 == 0 && TJ % 2 == 0, "even thread tiles");
  static_assert(KMODE ? (BK * BJ) % NTH == 0 : (BK * BJ) % (2 * NTH) == 0, "B loader coverage");
};

// One BM x BJ output tile of the step; `tile` enumerates (n tile, j tile) with the n tile
// fastest, `item` selects the batch entry.  NTH threads; `smem_raw` holds Cfg::SMEM bytes.
// Every output accumulates its k terms in the same order whatever the tile shape, so all
// variants give bit-identical results.
template <int BM, int BJ, int TM, int TJ, bool KMODE, int STAGES, int NTH = 256>
__device__ __forceinline__ void cgemm_tile(const StepArgs& a, int64_t tile, int64_t item,
                                           float4* smem_raw) {
  using C_ = Cfg<BM, BJ, TM, TJ, KMODE, STAGES, NTH>;
  constexpr int TXN = C_::TXN, LDA = C_::LDA, LDB = C_::LDB;
  float2* As = reinterpret_cast<float2*>(smem_raw);
  float2* Bs = As + STAGES * BK * LDA;

  const int tid = threadIdx.x;
  const int tx = tid % TXN, ty = tid / TXN;
  const int64_t NT = (a.N + BM - 1) / BM;
  const int64_t nt = tile % NT, jt = tile / NT;
  const int64_t n0 = nt * BM, j0 = jt * BJ;
  const float2* __restrict__ S = a.S + item * a.s_stride;
  const float2* __restrict__ B = a.B + item * a.b_stride;
  float2* __restrict__ C = a.C + item * a.c_stride;
  const int64_t K = a.K, N = a.N, Sd = a.Sd, J = a.J;

  // per-thread B source offsets (fixed for the whole k loop)
  int64_t boff[C_::B_IT];
  int bkk[C_::B_IT], bjj[C_::B_IT];
#pragma unroll
  for (int i = 0; i < C_::B_IT; ++i) {
    const int v = tid + i * NTH;
    if (KMODE) { bkk[i] = v % BK; bjj[i] = v / BK; }
    else       { bkk[i] = v / (BJ / 2); bjj[i] = (v % (BJ / 2)) * 2; }
    const int64_t j = j0 + bjj[i];
    boff[i] = j < J ? (j / Sd) * K * Sd + (j % Sd) : -1;
  }

  auto load_tile = [&](int stage, int64_t kt) {
    const int64_t k0 = kt * BK;
#pragma unroll
    for (int i = 0; i < C_::A_IT; ++i) {
      const int e = tid + i * NTH;
      if (e < BK * BM) {
        const int kk = e / BM, m = e % BM;
        const int64_t k = k0 + kk, n = n0 + m;
        const bool ok = k < K && n < N;
        cp_async8(&As[(stage * BK + kk) * LDA + m], ok ? S + k * N + n : S, ok);
      }
    }
#pragma unroll
    for (int i = 0; i < C_::B_IT; ++i) {
      const int64_t k = k0 + bkk[i];
      const bool ok = boff[i] >= 0 && k < K;
      const float2* src = ok ? B + boff[i] + k * Sd : B;
      if (KMODE) cp_async8(&Bs[(stage * BK + bkk[i]) * LDB + bjj[i]], src, ok);
      else       cp_async16(&Bs[(stage * BK + bkk[i]) * LDB + bjj[i]], src, ok);
    }
  };

  float accr[TM][TJ], acci[TM][TJ];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TJ; ++j) { accr[i][j] = 0.f; acci[i][j] = 0.f; }

  const int64_t KT = (K + BK - 1) / BK;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < KT) load_tile(s, s);
    cp_async_commit();
  }
  for (int64_t kt = 0; kt < KT; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    const int64_t nk = kt + STAGES - 1;
    if (nk < KT) load_tile((int)(nk % STAGES), nk);
    cp_async_commit();
    const int st = (int)(kt % STAGES);
    const float2* Ak = As + st * BK * LDA + ty * TM;
    const float2* Bk = Bs + st * BK * LDB + tx * 2;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 av[TM], bv[TJ];
#pragma unroll
      for (int i = 0; i < TM / 2; ++i) {
        const float4 t = *reinterpret_cast<const float4*>(Ak + kk * LDA + 2 * i);
        av[2 * i] = make_float2(t.x, t.y);
        av[2 * i + 1] = make_float2(t.z, t.w);
      }
#pragma unroll
      for (int c = 0; c < TJ / 2; ++c) {
        const float4 t = *reinterpret_cast<const float4*>(Bk + kk * LDB + c * 2 * TXN);
        bv[2 * c] = make_float2(t.x, t.y);
        bv[2 * c + 1] = make_float2(t.z, t.w);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          accr[i][j] = fmaf(av[i].x, bv[j].x, accr[i][j]);
          accr[i][j] = fmaf(-av[i].y, bv[j].y, accr[i][j]);
          acci[i][j] = fmaf(av[i].x, bv[j].y, acci[i][j]);
          acci[i][j] = fmaf(av[i].y, bv[j].x, acci[i][j]);
        }
    }
  }
  cp_async_wait<0>();

  // epilogue: C[nh][p][nl][s]
  const int64_t NL = a.NL;
  const int64_t strideNH = a.P * NL * Sd;
  // (nh, nl) of this thread's first row once; the rows below step with a carry (a 64-bit
  // division per element is a large share of the epilogue)
  const int nfirst = (int)(n0 + ty * TM), NLi = (int)NL;
  const int nh_first = nfirst / NLi, nl_first = nfirst % NLi;
#pragma unroll
  for (int c = 0; c < TJ / 2; ++c) {
    const int64_t j = j0 + c * 2 * TXN + tx * 2;
    if (j >= J) continue;
    const int64_t p = j / Sd, s = j % Sd;
    const int64_t p1 = (j + 1) / Sd, s1 = (j + 1) % Sd;
    int nh = nh_first, nl = nl_first;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t n = nfirst + i;
      if (n >= N) break;
      if (i > 0 && ++nl == NLi) { nl = 0; ++nh; }
      const float2 v0 = make_float2(accr[i][2 * c], acci[i][2 * c]);
      const float2 v1 = make_float2(accr[i][2 * c + 1], acci[i][2 * c + 1]);
      float2* dst0 = C + nh * strideNH + p * (NL * Sd) + nl * Sd + s;
      if (!KMODE) {
        float4 w = make_float4(v0.x, v0.y, v1.x, v1.y);
        if (a.beta) {
          const float4 o = *reinterpret_cast<const float4*>(dst0);
          w.x += o.x; w.y += o.y; w.z += o.z; w.w += o.w;
        }
        *reinterpret_cast<float4*>(dst0) = w;
      } else {
        float2 w0 = v0;
        if (a.beta) { w0.x += dst0->x; w0.y += dst0->y; }
        *dst0 = w0;
        if (j + 1 < J) {
          float2* dst1 = C + nh * strideNH + p1 * (NL * Sd) + nl * Sd + s1;
          float2 w1 = v1;
          if (a.beta) { w1.x += dst1->x; w1.y += dst1->y; }
          *dst1 = w1;
        }
      }
    }
  }
}


// Tile variants: 0..4 stream B along s (JMODE), 5..9 the same tiles loading B along k.
#define QFX_SIMT_VARIANTS(X)               \
  X(0, 128, 128, 8, 8, false, 3)           \
  X(1, 64, 256, 8, 8, false, 3)            \
  X(2, 32, 512, 8, 8, false, 3)            \
  X(3, 16, 512, 8, 4, false, 3)            \
  X(4, 8, 512, 8, 2, false, 3)             \
  X(5, 128, 128, 8, 8, true, 3)            \
  X(6, 64, 256, 8, 8, true, 3)             \
  X(7, 32, 512, 8, 8, true, 3)             \
  X(8, 16, 512, 8, 4, true, 3)             \
  X(9, 8, 512, 8, 2, true, 3)

// Fill variants: the same tiles with a quarter (or half) of the outputs per CTA, 4 x 4 (or
// 4 x 2) per thread, for grids that the tiles above would leave with fewer CTAs than two
// per SM (fill_variant picks them at launch time; the batch scheduler keeps 0..9).
// Variants 0, 1, 2, 3, 4 map to 20, 20, 21, 22, 23 and 5..9 to 25, 25, 26, 27, 28; the last
// argument is the CTA's thread count.
#define QFX_SIMT_FILL_VARIANTS(X)          \
  X(20, 64, 64, 4, 4, false, 3, 256)       \
  X(21, 32, 128, 4, 4, false, 3, 256)      \
  X(22, 16, 256, 4, 4, false, 3, 256)      \
  X(23, 8, 256, 4, 2, false, 3, 256)       \
  X(25, 64, 64, 4, 4, true, 3, 256)        \
  X(26, 32, 128, 4, 4, true, 3, 256)       \
  X(27, 16, 256, 4, 4, true, 3, 256)       \
  X(28, 8, 256, 4, 2, true, 3, 256)

}  // namespace simt
}  // namespace qfx
