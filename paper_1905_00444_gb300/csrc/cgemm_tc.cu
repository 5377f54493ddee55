// One contraction step on the 5th-generation tensor cores (tcgen05, TMEM accumulators),
// with complex FP32 operands split into lower-precision terms.
//
//   C[nh][p][nl][s] = sum_k S[k][nh*NL + nl] * B[p][k][s]     (Sec. III.E, Eq. 1)
//
// The paper ran this product as complex FP32 CGEMM without tensor cores, because FP16
// inputs lose too much precision (Sec. III.E).  Here each FP32 real operand x is split
// into terms of a tensor-core type and the complex product is formed from real products
// (4M: Re = Ar Sr - Ai Si, Im = Ar Si + Ai Sr), each real product being the sum of the
// cross products of the terms whose magnitude is above FP32 rounding:
//   BF16x3: x = h + m + l (successive round-to-nearest residuals), products
//           hh, hm, mh, hl, lh, mm  (error ~2^-24 relative);
//   TF32x3: x = b + s, products bb, bs, sb  (error ~2^-21 relative).
// Accumulation is FP32 in TMEM.
//
// Tiles: a persistent CTA per SM walks tiles of 128 columns j (M = 128; the boundary
// tensor B is the A operand, rows j) by Nt rows n of the site matrix S (the B operand).
// Default tiles are 128 x 128 with split accumulators in TMEM: hi x hi products go to
// "main" accumulators (re [0,128), im [128,256)), every cross-term product to "small"
// ones (re [256,384), im [384,512)), added in the epilogue, so the large accumulators
// see two additions per k-stage.  There the complex product is embedded in N: S is held
// per term as planes Sr, Si, -Sr, and one MMA of N = 256 takes Ar x [Sr; Si] into
// (re, im) and another -Ai x [Si; -Sr], so each MMA reads A once for both halves.
// QFX_TC_FAST_ACCUMULATION tiles are 128 x 256 with one accumulator pair
// (re [0,256), im [256,512)) and four real products per term pair (4M).
// Roles (14 warps):
//   warps 0-3   producers: FP32 rows of B -> term planes in shared memory (K-major,
//               no-swizzle core-matrix layout).  Default tiles take the rows from
//               staging buffers filled by tensor-map copies (cp.async.bulk.tensor) when
//               the shape allows it, otherwise they load them one k-stage ahead;
//   warps 4-11  epilogue: TMEM -> registers -> C (two warps per TMEM lane quarter);
//   warp 12     allocates TMEM; lane 0 issues tcgen05.mma;
//   warp 13     lane 0 streams the pre-split image of S (written once per step by
//               split_site_kernel in the same layout) with one bulk copy per stage;
//               lane 1 issues the tensor-map copies of B.
// Rings of shared-memory stages are guarded by mbarriers.  Every wait has a deadline;
// on expiry the kernel records an error, drains its own copies and MMAs, frees TMEM and
// returns (the host reports QFX_ETIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "ptx_async.cuh"
#include "qfx_internal.h"

namespace qfx {

__device__ unsigned int g_tc_status = 0;

namespace {

using namespace ptx;

constexpr int kRows = 128;        // UMMA M
constexpr int kPlaneA = kRows * 32;   // bytes of one A term plane per stage
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s per wait

template <int MODE>
struct Mode;
template <>
struct Mode<QFX_PREC_C3M_BF16X3> {
  static constexpr int TERMS = 3, KS = 16, NPROD = 6;
  static constexpr uint32_t FMT = 1;   // BF16
  __device__ static constexpr int ta(int i) { return i == 0 ? 1 : i == 1 ? 0 : i == 2 ? 2 : i == 3 ? 0 : i == 4 ? 1 : 0; }
  __device__ static constexpr int tb(int i) { return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 0 : i == 3 ? 1 : i == 4 ? 0 : 0; }
};
template <>
struct Mode<QFX_PREC_C3M_BF16X2> {
  static constexpr int TERMS = 2, KS = 16, NPROD = 3;
  static constexpr uint32_t FMT = 1;   // BF16: h, m with products hm, mh, hh (~2^-16)
  __device__ static constexpr int ta(int i) { return i == 0 ? 0 : i == 1 ? 1 : 0; }
  __device__ static constexpr int tb(int i) { return i == 0 ? 1 : i == 1 ? 0 : 0; }
};
template <>
struct Mode<QFX_PREC_C3M_TF32X3> {
  static constexpr int TERMS = 2, KS = 8, NPROD = 3;
  static constexpr uint32_t FMT = 2;   // TF32
  __device__ static constexpr int ta(int i) { return i == 0 ? 0 : i == 1 ? 1 : 0; }
  __device__ static constexpr int tb(int i) { return i == 0 ? 1 : i == 1 ? 0 : 0; }
};

// ---- term splitting ------------------------------------------------------------
// T BF16 terms of x: each the round-to-nearest of what the previous ones left
template <int T>
__device__ __forceinline__ void split_bf16(float x, uint16_t t[T]) {
  float r = x;
#pragma unroll
  for (int i = 0; i < T; ++i) {
    const __nv_bfloat16 h = __float2bfloat16_rn(r);
    t[i] = __bfloat16_as_ushort(h);
    r -= __bfloat162float(h);
  }
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32x2(float x, uint32_t t[2]) {
  t[0] = to_tf32(x);
  t[1] = to_tf32(x - __uint_as_float(t[0]));
}

// Writes the KS values of one row (component c of `v`) as TERMS planes of 32 bytes each.
// Row r of a plane lives at (r/8)*256 + kc*128 + (r%8)*16 (8x16-byte core matrices;
// kc = which 16-byte half of the row).
template <int MODE>
__device__ __forceinline__ void store_row_terms(char* plane0, int plane_bytes, int row,
                                                const float* x) {
  using M_ = Mode<MODE>;
  const int base = (row >> 3) * 256 + (row & 7) * 16;
  if constexpr (M_::FMT == 1) {   // BF16 terms, 16 per row
    constexpr int T = M_::TERMS;
    uint32_t w[T][8];
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
      uint16_t a[T], b[T];
      split_bf16<T>(x[k], a);
      split_bf16<T>(x[k + 1], b);
#pragma unroll
      for (int t = 0; t < T; ++t) w[t][k / 2] = (uint32_t)a[t] | ((uint32_t)b[t] << 16);
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
      char* pl = plane0 + t * plane_bytes + base;
      *reinterpret_cast<uint4*>(pl) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
      *reinterpret_cast<uint4*>(pl + 128) = make_uint4(w[t][4], w[t][5], w[t][6], w[t][7]);
    }
  } else {
    uint32_t w[2][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t a[2];
      split_tf32x2(x[k], a);
      w[0][k] = a[0];
      w[1][k] = a[1];
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      char* pl = plane0 + t * plane_bytes + base;
      *reinterpret_cast<uint4*>(pl) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
      *reinterpret_cast<uint4*>(pl + 128) = make_uint4(w[t][4], w[t][5], w[t][6], w[t][7]);
    }
  }
  (void)sizeof(M_);
}

// ---- PTX helpers -----------------------------------------------------------------
// Bounded wait: false if the deadline passed or another role gave up.  Roles off the
// critical path pass sleep_ns > 0 so that their polling does not take issue slots from
// the producers.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          unsigned sleep_ns = 0) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long deadline = globaltimer() + kWaitNs;
  while (!mbar_try(bar, parity)) {
    if (*abort) return false;
    if (globaltimer() > deadline) {
      *abort = 1;
      atomicOr(&g_tc_status, 1u);
      return false;
    }
    if (sleep_ns) __nanosleep(sleep_ns);
  }
  return true;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  // K-major, no swizzle: LBO = 128 B (next core matrix along K), SBO = 256 B (next
  // 8-row group); bits 46-48 = 0b001; base offset 0; layout type 0.
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}
template <int MODE>
__device__ __forceinline__ uint32_t instr_desc(int n, bool neg_a) {
  // D = F32 (bits 4-5 = 1), A/B format (bits 7-9, 10-12), negate A (bit 13),
  // both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
  return (1u << 4) | (Mode<MODE>::FMT << 7) | (Mode<MODE>::FMT << 10) | ((neg_a ? 1u : 0u) << 13) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}
template <int MODE>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (MODE == QFX_PREC_C3M_BF16X3) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  const float2* B; int64_t b_stride;
  float2* C; int64_t c_stride;
  const char* simage; int64_t img_stride;   // pre-split S, per item
  int64_t P, K, N, NL, Sd, J;
  int Nt;            // columns n per tile (<= 128 split accumulators, <= 256 single)
  int NHt;           // tiles along n per 128-row tile
  int64_t JT;        // 128-row tiles per item
  int64_t tiles;     // total tiles (items x JT x NHt)
  int withhold_s;    // test hook: never stream S, so the bounded waits expire
  int use_tma;       // producers read FP32 rows staged by tensor-map copies (default tiles)
  int box_s, box_p;  // tensor-map box: box_s consecutive s (columns), box_p values of p
  int beta;          // 1: add the product into C (a chunk of a long contraction)
};

// Persistent CTA, one per SM.  TMEM columns: with SPLITACC the hh-term products go to
// "main" accumulators (re [0,Nt), im [Nt,2Nt)) and every cross-term product to "small"
// ones (re [256,256+Nt), im [256+Nt,256+2Nt)), so the large accumulator sees 2 additions
// per k-stage instead of 2 x NPROD; without SPLITACC re = [0, Nt), im = [256, 256 + Nt).
// Warps: 0-3 producers, 4-11 epilogue (two per TMEM lane quarter, each half the columns),
// 12 TMEM owner + MMA issuer, 13 S stream and tensor-map copies.
constexpr uint32_t kAlignPad = 128;

// Tile t -> (item g, 128-row tile jt, column tile nh).  Within an item the column tiles
// come in bands of kBand; inside a band the column tile runs fastest, so the tiles in
// flight at once (one per CTA) share a few column slices of the S image and a few row
// tiles of B in L2 (with N = 8192 one k-chunk of the S image alone is 151 MB).  With
// NHt <= kBand this is the plain order, column tile fastest.
constexpr int64_t kBand = 8;
__device__ __forceinline__ void tile_coords(const TcArgs& a, int64_t t, int64_t& g, int64_t& jt,
                                            int64_t& nh) {
  const int64_t per_item = a.JT * a.NHt;
  g = t / per_item;
  int64_t r = t - g * per_item;
  const int64_t band = r / (kBand * a.JT);
  const int64_t n0 = band * kBand;
  const int64_t w = a.NHt - n0 < kBand ? a.NHt - n0 : kBand;
  r -= band * kBand * a.JT;
  jt = r / w;
  nh = n0 + (r - jt * w);
}

template <int MODE, bool SPLITACC>
struct TcCfg {
  using M_ = Mode<MODE>;
  static constexpr int NT_MAX = SPLITACC ? 128 : 256;
  // default tiles hold S as [Sr; Si; -Sr] per term (the complex product embedded in N)
  static constexpr int PLANES = 2 * M_::TERMS;             // A planes per stage
  static constexpr int SPLANES = SPLITACC ? 3 * M_::TERMS : PLANES;   // S planes per stage
  static constexpr int STAGES = SPLITACC ? (M_::TERMS == 3 ? 3 : 4) : 3;
  static constexpr int STAGE_A = PLANES * kPlaneA;
  static constexpr int THREADS = 14 * 32;
  // FP32 rows of the default tile arrive by tensor-map copies into NBUF staging buffers;
  // the fast tile's operand ring leaves no room and keeps register prefetch
  static constexpr int STAGE_IN = kRows * M_::KS * 8;
  static constexpr int NBUF = SPLITACC ? (M_::KS == 16 ? 2 : 4) : 0;
  static size_t smem(int nt) {
    return kAlignPad + (size_t)STAGES * (STAGE_A + SPLANES * nt * 32) + (size_t)NBUF * STAGE_IN +
           (3 * STAGES + 3 + 2 * NBUF) * sizeof(uint64_t);
  }
};

template <int MODE, bool SPLITACC>
__global__ void __launch_bounds__(TcCfg<MODE, SPLITACC>::THREADS, 1)
    cgemm_tc_kernel(const TcArgs a, const __grid_constant__ CUtensorMap tmA) {
  using M_ = Mode<MODE>;
  using CF = TcCfg<MODE, SPLITACC>;
  constexpr int TERMS = M_::TERMS, KS = M_::KS, STAGES = CF::STAGES;
  extern __shared__ __align__(16) char smem_raw[];
  // tensor-map copies land on 128-byte boundaries; the dynamic window itself is only
  // 16-byte aligned behind the static shared variables
  char* smem = smem_raw + ((kAlignPad - (smem_u32(smem_raw) & (kAlignPad - 1))) & (kAlignPad - 1));
  const int stageA = CF::STAGE_A;
  const int planeS = a.Nt * 32;
  const int stageS = CF::SPLANES * planeS;
  char* sA = smem;
  char* sS = smem + STAGES * stageA;
  char* sIn = sS + STAGES * stageS;                 // NBUF x [box_p][KS][box_s] float2
  uint64_t* bars = reinterpret_cast<uint64_t*>(sIn + CF::NBUF * CF::STAGE_IN);
  // bars: fullA[S], fullS[S], empty[S], acc_full, tmem_free, done, in_full[NBUF], in_empty[NBUF]
  __shared__ uint32_t tmem_base_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t KT = a.K / KS;

  auto fullA = [&](int s) { return smem_u32(&bars[s]); };
  auto fullS = [&](int s) { return smem_u32(&bars[STAGES + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * STAGES + s]); };
  const uint32_t acc_full = smem_u32(&bars[3 * STAGES]);
  const uint32_t tmem_free = smem_u32(&bars[3 * STAGES + 1]);
  const uint32_t done = smem_u32(&bars[3 * STAGES + 2]);
  auto in_full = [&](int b) { return smem_u32(&bars[3 * STAGES + 3 + b]); };
  auto in_empty = [&](int b) { return smem_u32(&bars[3 * STAGES + 3 + CF::NBUF + b]); };

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(fullA(s), kRows);
      mbar_init(fullS(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(tmem_free, 8);
    mbar_init(done, 1);
    for (int b = 0; b < CF::NBUF; ++b) {
      mbar_init(in_full(b), 1);
      mbar_init(in_empty(b), kRows);
    }
    mbar_init_fence();
  }
  if (warp == 12) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;
  volatile int* abort = &abort_flag;

  if (warp < 4) {
    // ---- producers: split 128 rows of B per k-stage into term planes -------------------
    // Rows arrive either through tensor-map copies staged NBUF k-stages ahead (default
    // tiles, issued by warp 13) or through loads issued one k-stage ahead into registers,
    // so their latency overlaps the split and the wait for a free operand stage.
    int64_t t = blockIdx.x, it = 0, q = 0;
    if (CF::NBUF > 0 && a.use_tma) {
      const int ps = tid / a.box_s, ss = tid % a.box_s;     // this row inside the box
      while (t < a.tiles && !*abort) {
        const int b = (int)(q % (CF::NBUF > 0 ? CF::NBUF : 1));
        if (!mbar_wait(in_full(b), (uint32_t)((q / (CF::NBUF > 0 ? CF::NBUF : 1)) & 1), abort)) break;
        const float2* in = reinterpret_cast<const float2*>(sIn + b * CF::STAGE_IN);
        float re[KS], im[KS];
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
          const float2 v = in[(ps * KS + kk) * a.box_s + ss];
          re[kk] = v.x;
          im[kk] = v.y;
        }
        // the next tensor-map copy rewrites this buffer through the async proxy: order
        // these generic reads before it (without the fence, fast consumers saw rows of the
        // following k-stage)
        fence_async_smem();
        mbar_arrive(in_empty(b));
        const int s = (int)(q % STAGES);
        if (q >= STAGES && !mbar_wait(empty(s), (uint32_t)((q / STAGES - 1) & 1), abort)) break;
        char* st = sA + s * stageA;
        store_row_terms<MODE>(st, kPlaneA, tid, re);
        store_row_terms<MODE>(st + TERMS * kPlaneA, kPlaneA, tid, im);
        fence_async_smem();
        mbar_arrive(fullA(s));
        ++q;
        if (++it == KT) { it = 0; t += gridDim.x; }
      }
    } else {
    auto row_ptr = [&](int64_t tt, int64_t& pofs) -> const float2* {
      int64_t g, jt, nh;
      tile_coords(a, tt, g, jt, nh);
      const int64_t jg = jt * kRows + tid;
      pofs = jg < a.J ? (jg / a.Sd) * a.K * a.Sd + (jg % a.Sd) : -1;
      return a.B + g * a.b_stride;
    };
    float2 nxt[KS];
    auto fetch = [&](int64_t tt, int64_t ii) {
      int64_t pofs;
      const float2* Bg = row_ptr(tt, pofs);
#pragma unroll
      for (int kk = 0; kk < KS; ++kk)
        nxt[kk] = pofs >= 0 ? __ldg(Bg + pofs + (ii * KS + kk) * a.Sd) : make_float2(0.f, 0.f);
    };
    if (t < a.tiles) fetch(t, 0);
    while (t < a.tiles && !*abort) {
      float re[KS], im[KS];
#pragma unroll
      for (int kk = 0; kk < KS; ++kk) { re[kk] = nxt[kk].x; im[kk] = nxt[kk].y; }
      int64_t nt = t, ni = it + 1;
      if (ni == KT) { nt = t + gridDim.x; ni = 0; }
      if (nt < a.tiles) fetch(nt, ni);
      const int s = (int)(q % STAGES);
      if (q >= STAGES && !mbar_wait(empty(s), (uint32_t)((q / STAGES - 1) & 1), abort)) break;
      char* st = sA + s * stageA;
      store_row_terms<MODE>(st, kPlaneA, tid, re);
      store_row_terms<MODE>(st + TERMS * kPlaneA, kPlaneA, tid, im);
      fence_async_smem();
      mbar_arrive(fullA(s));
      ++q;
      t = nt;
      it = ni;
    }
    }
  } else if (warp == 13) {
    // ---- S image stream ------------------------------------------------------------
    if (lane == 0) {
      int64_t q = 0, issued = 0;
      bool ok = !a.withhold_s;
      for (int64_t t = blockIdx.x; t < a.tiles && ok; t += gridDim.x) {
        int64_t g, jt, nh;
        tile_coords(a, t, g, jt, nh);
        const char* img = a.simage + g * a.img_stride;
        for (int64_t it = 0; it < KT; ++it, ++q) {
          const int s = (int)(q % STAGES);
          if (q >= STAGES && !mbar_wait(empty(s), (uint32_t)((q / STAGES - 1) & 1), abort, 32)) { ok = false; break; }
          mbar_arrive_tx(fullS(s), (uint32_t)stageS);
          bulk_copy(smem_u32(sS + s * stageS), img + (it * a.NHt + nh) * stageS, (uint32_t)stageS, fullS(s));
          issued = q + 1;
        }
      }
      // drain: every issued copy must land before the CTA exits
      for (int64_t i = (issued > STAGES ? issued - STAGES : 0); i < issued; ++i) {
        const int s = (int)(i % STAGES);
        const unsigned long long deadline = globaltimer() + kWaitNs;
        while (!mbar_try(fullS(s), (uint32_t)((i / STAGES) & 1)) && globaltimer() < deadline) {
        }
      }
    } else if (lane == 1 && CF::NBUF > 0 && a.use_tma) {
      // ---- FP32 rows of B: one tensor-map copy per (tile, k-stage) into staging --------
      constexpr int NB = CF::NBUF > 0 ? CF::NBUF : 1;
      int64_t q = 0, issued = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < a.tiles && ok; t += gridDim.x) {
        int64_t g, jt, nh;
        tile_coords(a, t, g, jt, nh);
        const int64_t j0 = jt * kRows;
        const int c0 = (int)(j0 % a.Sd), c2 = (int)(j0 / a.Sd);
        for (int64_t it = 0; it < KT; ++it, ++q) {
          const int b = (int)(q % NB);
          if (q >= NB && !mbar_wait(in_empty(b), (uint32_t)((q / NB - 1) & 1), abort, 32)) { ok = false; break; }
          mbar_arrive_tx(in_full(b), (uint32_t)CF::STAGE_IN);
          tma_load_4d(smem_u32(sIn + b * CF::STAGE_IN), &tmA, c0, (int)(it * KS), c2, (int)g, in_full(b));
          issued = q + 1;
        }
      }
      for (int64_t i = (issued > NB ? issued - NB : 0); i < issued; ++i) {
        const int b = (int)(i % NB);
        const unsigned long long deadline = globaltimer() + kWaitNs;
        while (!mbar_try(in_full(b), (uint32_t)((i / NB) & 1)) && globaltimer() < deadline) {
        }
      }
    }
  } else if (warp == 12) {
    // ---- MMA issue -----------------------------------------------------------------
    if (lane == 0) {
      int64_t q = 0, tc = 0;
      bool ok = true;
      // default tiles: one MMA covers re and im (N = 2 Nt); fast tiles: N = Nt
      const int n_mma = SPLITACC ? 2 * a.Nt : a.Nt;
      const uint32_t idesc_p = instr_desc<MODE>(n_mma, false), idesc_n = instr_desc<MODE>(n_mma, true);
      for (int64_t t = blockIdx.x; t < a.tiles && ok; t += gridDim.x, ++tc) {
        if (tc > 0 && !mbar_wait(tmem_free, (uint32_t)((tc - 1) & 1), abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool started[2] = {false, false};
        for (int64_t it = 0; it < KT; ++it, ++q) {
          const int s = (int)(q % STAGES);
          const uint32_t par = (uint32_t)((q / STAGES) & 1);
          if (!mbar_wait(fullA(s), par, abort) || !mbar_wait(fullS(s), par, abort)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * stageA), b0 = smem_u32(sS + s * stageS);
          if constexpr (SPLITACC) {
            // Ar x [Sr; Si] -> (re, im) += (Ar Sr, Ar Si);  (-Ai) x [Si; -Sr] -> += (-Ai Si, Ai Sr)
#pragma unroll
            for (int ca = 0; ca < 2; ++ca) {
#pragma unroll
              for (int pi = 0; pi < M_::NPROD; ++pi) {
                const bool main_term = M_::ta(pi) == 0 && M_::tb(pi) == 0;
                const int acc = main_term ? 0 : 1;
                const uint64_t ad = smem_desc(a0 + (ca * TERMS + M_::ta(pi)) * kPlaneA);
                const uint64_t bd = smem_desc(b0 + (3 * M_::tb(pi) + ca) * planeS);
                mma<MODE>(tmem + (uint32_t)(acc * 256), ad, bd, ca ? idesc_n : idesc_p, started[acc] ? 1u : 0u);
                started[acc] = true;
              }
            }
          } else {
            // 4M with re in TMEM columns [0, Nt) and im in [256, 256 + Nt)
#pragma unroll
            for (int rp = 0; rp < 4; ++rp) {
              const int ca = (rp == 0 || rp == 2) ? 0 : 1;          // Ar, Ai, Ar, Ai
              const int cb = (rp == 0 || rp == 3) ? 0 : 1;          // Sr, Si, Si, Sr
              const int to_im = rp >= 2 ? 1 : 0;
              const uint32_t idesc = rp == 1 ? idesc_n : idesc_p;   // - Ai Si
#pragma unroll
              for (int pi = 0; pi < M_::NPROD; ++pi) {
                const uint64_t ad = smem_desc(a0 + (ca * TERMS + M_::ta(pi)) * kPlaneA);
                const uint64_t bd = smem_desc(b0 + (cb * TERMS + M_::tb(pi)) * planeS);
                mma<MODE>(tmem + (uint32_t)(to_im * 256), ad, bd, idesc, started[to_im] ? 1u : 0u);
                started[to_im] = true;
              }
            }
          }
          mma_commit(empty(s));
        }
        if (ok) mma_commit(acc_full);
      }
      mma_commit(done);
    }
  } else {
    // ---- epilogue (warps 4-11): TMEM -> C ----------------------------------------------
    const int quarter = warp & 3, half = (warp - 4) >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    // 16-column chunks alternate between the two warps of a lane quarter
    const int nchunks = a.Nt / 16;
    const int my_last = ((nchunks - 1 - half) >= 0) ? (nchunks - 1 - ((nchunks - 1 - half) & 1)) : -1;
    int64_t tc = 0;
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x, ++tc) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_full, (uint32_t)(tc & 1), abort, 256) && !*abort);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int64_t g, jt, nh;
      tile_coords(a, t, g, jt, nh);
      const int64_t jg = jt * kRows + row;
      const bool valid = jg < a.J;
      float2* Cg = a.C + g * a.c_stride;
      const int64_t p = valid ? jg / a.Sd : 0, sidx = valid ? jg % a.Sd : 0;
      const int64_t jofs = p * a.NL * a.Sd + sidx;
      const int64_t strideNH = a.P * a.NL * a.Sd;
      if (my_last < 0) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(tmem_free);
      }
      for (int ci = half; ci < nchunks; ci += 2) {
        const int c0 = ci * 16;
        float vr[16], vi[16];
        if (SPLITACC) {
          // main (re, im) in columns [0, Nt), [Nt, 2 Nt); small ones 256 further
          float sr[16], si[16];
          tmem_ld16(tmem + lane_base + c0, vr);
          tmem_ld16(tmem + lane_base + a.Nt + c0, vi);
          tmem_ld16(tmem + lane_base + 256 + c0, sr);
          tmem_ld16(tmem + lane_base + 256 + a.Nt + c0, si);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 16; ++i) { vr[i] += sr[i]; vi[i] += si[i]; }
        } else {
          tmem_ld16(tmem + lane_base + c0, vr);
          tmem_ld16(tmem + lane_base + 256 + c0, vi);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
        if (ci == my_last) {
          // last TMEM read of this tile by this warp: hand the columns back to the MMA
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(tmem_free);
        }
        if (valid) {
          // one division per chunk, then step along n with a carry into nh (a 64-bit
          // division per element cost more than the MMAs of the tile)
          const int n0 = (int)nh * a.Nt + c0, NL = (int)a.NL;
          int nl = n0 % NL;
          float2* dst = Cg + (int64_t)(n0 / NL) * strideNH + (int64_t)nl * a.Sd + jofs;
          if (!a.beta) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              *dst = make_float2(vr[i], vi[i]);
              dst += a.Sd;
              if (++nl == NL) { nl = 0; dst += strideNH - (int64_t)NL * a.Sd; }
            }
          } else {   // a chunk of a long contraction: add into C
            // all 16 reads first (C is written only by this tile in this launch, so the
            // read-only path applies): one memory latency per chunk, not one per element
            float2 o[16];
            float2* d = dst;
            int l = nl;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              o[i] = __ldg(d);
              d += a.Sd;
              if (++l == NL) { l = 0; d += strideNH - (int64_t)NL * a.Sd; }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              *dst = make_float2(vr[i] + o[i].x, vi[i] + o[i].y);
              dst += a.Sd;
              if (++nl == NL) { nl = 0; dst += strideNH - (int64_t)NL * a.Sd; }
            }
          }
        }
      }
    }
  }

  if (warp == 12) mbar_wait(done, 0, abort, 256);   // last MMAs finished before freeing TMEM
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 12) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Pre-split of the site matrix S[k][n] into the per-stage shared-memory image, per
// (stage ks, n tile), each plane [row n within the tile][32 bytes]:
//   EMB (default tiles): per term t the planes Sr_t, Si_t, -Sr_t, so that [Sr_t; Si_t]
//     and [Si_t; -Sr_t] are contiguous 2 Nt-row operands (complex product embedded in N);
//   otherwise: Sr terms then Si terms.
template <int MODE, bool EMB>
__global__ void __launch_bounds__(128) split_site_kernel(const float2* __restrict__ S, int64_t s_stride,
                                                          int K, int N, int Nt, char* image,
                                                          int64_t img_stride) {
  using M_ = Mode<MODE>;
  constexpr int TERMS = M_::TERMS, KS = M_::KS;
  const int n = blockIdx.x * 128 + threadIdx.x;
  const int ks = blockIdx.y;
  const int g = blockIdx.z;
  if (n >= N) return;
  const float2* Sg = S + (int64_t)g * s_stride;
  float re[KS], im[KS];
#pragma unroll
  for (int kk = 0; kk < KS; ++kk) {
    const int k = ks * KS + kk;
    float2 v = make_float2(0.f, 0.f);
    if (k < K) v = Sg[(int64_t)k * N + n];
    re[kk] = v.x;
    im[kk] = v.y;
  }
  const int planeS = Nt * 32;
  const int nht = N / Nt, nh = n / Nt, r = n % Nt;
  constexpr int SPL = EMB ? 3 * TERMS : 2 * TERMS;
  char* st = image + (int64_t)g * img_stride + ((int64_t)ks * nht + nh) * SPL * planeS;
  if constexpr (EMB) {
    store_row_terms<MODE>(st, 3 * planeS, r, re);
    store_row_terms<MODE>(st + planeS, 3 * planeS, r, im);
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) re[kk] = -re[kk];
    store_row_terms<MODE>(st + 2 * planeS, 3 * planeS, r, re);
  } else {
    store_row_terms<MODE>(st, planeS, r, re);
    store_row_terms<MODE>(st + TERMS * planeS, planeS, r, im);
  }
}

// Tensor map over B viewed as (s, k, p, item) 8-byte elements, box (box_s, KS, box_p, 1)
// = one 128-row, KS-deep k-stage of a tile.  False if the shape does not allow it (the
// box's inner extent must be at least 16 bytes: Sd >= 2; tiles must not straddle p
// unevenly: Sd a multiple of 128 or a divisor of it).
bool make_b_map(CUtensorMap* map, const void* B, int64_t b_stride, int batch, int64_t P, int64_t K,
                int64_t Sd, int ks, int* box_s, int* box_p) {
  auto enc = tensor_map_encoder();
  if (!enc || Sd < 2 || (Sd % 128 != 0 && 128 % Sd != 0)) return false;
  const int bs = (int)(Sd < 128 ? Sd : 128), bp = 128 / bs;
  const cuuint64_t dims[4] = {(cuuint64_t)Sd, (cuuint64_t)K, (cuuint64_t)P, (cuuint64_t)batch};
  const cuuint64_t item = (cuuint64_t)(batch > 1 ? b_stride : P * K * Sd) * 8;
  const cuuint64_t strides[3] = {(cuuint64_t)Sd * 8, (cuuint64_t)(K * Sd) * 8, item};
  const cuuint32_t box[4] = {(cuuint32_t)bs, (cuuint32_t)ks, (cuuint32_t)bp, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (((uintptr_t)B & 15) || (item & 15)) return false;
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(B), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  *box_s = bs;
  *box_p = bp;
  return true;
}

// Shared-memory opt-in of one tensor-core kernel, once per device (also called ahead of a
// graph capture).
template <int MODE, bool SPLITACC>
int ensure_tc_attr() {
  using CF = TcCfg<MODE, SPLITACC>;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_tc_kernel<MODE, SPLITACC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CF::smem(CF::NT_MAX));
    if (e != cudaSuccess) return (int)e;
    attr_done[dev] = 1;
  }
  return 0;
}

template <int MODE, bool SPLITACC>
int launch_tc_mode(const void* S, int64_t s_stride, const void* B, int64_t b_stride, void* C,
                   int64_t c_stride, int64_t P, int64_t K, int64_t N, int64_t NL, int64_t Sd,
                   int batch, char* scratch, int64_t scratch_stride, int withhold, bool no_tma, int beta,
                   cudaStream_t st) {
  using M_ = Mode<MODE>;
  using CF = TcCfg<MODE, SPLITACC>;
  const int Nt = (int)(N < CF::NT_MAX ? N : CF::NT_MAX);   // N % 16 == 0, N <= 256
  const int KT = (int)(K / M_::KS);
  dim3 sg((unsigned)((N + 127) / 128), KT, batch);
  split_site_kernel<MODE, SPLITACC><<<sg, 128, 0, st>>>((const float2*)S, s_stride, (int)K, (int)N, Nt,
                                              scratch, scratch_stride);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  TcArgs a{};
  a.B = (const float2*)B; a.b_stride = b_stride;
  a.C = (float2*)C; a.c_stride = c_stride;
  a.simage = scratch; a.img_stride = scratch_stride;
  a.P = P; a.K = K; a.N = N; a.NL = NL; a.Sd = Sd; a.J = P * Sd;
  a.Nt = Nt;
  a.NHt = (int)(N / Nt);
  a.JT = (a.J + kRows - 1) / kRows;
  a.tiles = (int64_t)batch * a.JT * a.NHt;
  a.withhold_s = withhold;
  a.beta = beta;
  alignas(64) CUtensorMap tmA;
  std::memset(&tmA, 0, sizeof(tmA));
  a.use_tma = 0;
  if (CF::NBUF > 0 && !no_tma)
    a.use_tma = make_b_map(&tmA, B, b_stride, batch, P, K, Sd, M_::KS, &a.box_s, &a.box_p) ? 1 : 0;
  auto kern = cgemm_tc_kernel<MODE, SPLITACC>;
  if (int err = ensure_tc_attr<MODE, SPLITACC>()) return err;
  const int64_t grid = a.tiles < num_sms() ? a.tiles : num_sms();
  kern<<<(unsigned)grid, CF::THREADS, CF::smem(Nt), st>>>(a, tmA);
  count_launch();
  return (int)cudaGetLastError();
}

// ---- tensor-core rate probe -------------------------------------------------------
// One CTA per SM (its shared-memory request leaves room for no second one) issues `iters`
// MMAs of the mode's operand kind, M = 128, N = 256, one K step, from fixed pseudo-random
// shared-memory operands into two alternating TMEM accumulators, committing every 256
// MMAs.  The host times the launch: dense tensor flop/s of that kind as this code issues it.
constexpr size_t kProbeSmem = 128 << 10;
template <int MODE>
__global__ void __launch_bounds__(128, 1) tc_probe_kernel(int64_t iters) {
  extern __shared__ __align__(16) char probe_raw[];
  char* sm = probe_raw + ((128u - (smem_u32(probe_raw) & 127u)) & 127u);
  char* sA = sm;               // 128 rows x 32 B
  char* sB = sm + kPlaneA;     // 256 rows x 32 B
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  // operands: 12 KB of small pseudo-random values of the mode's type
  for (int i = tid; i < 3 * kPlaneA / 4; i += blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u + 0x9e3779b9u * (blockIdx.x + 1);
    h ^= h >> 15;
    const float x = (float)(h & 0xffff) * (1.0f / 65536.0f) - 0.5f;
    uint32_t w;
    if constexpr (Mode<MODE>::FMT == 1) {
      const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
      w = b | (b << 16);
    } else {
      w = __float_as_uint(x) & 0xffffe000u;   // TF32: 10 explicit mantissa bits
    }
    reinterpret_cast<uint32_t*>(sm)[i] = w;
  }
  fence_async_smem();
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    mbar_init_fence();
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid < 32) {
    // warp-uniform loop; lane 0 issues 16 MMAs per iteration (a thread issuing one MMA per
    // loop iteration kept the tensor pipe about half idle)
    volatile int* abort = &abort_flag;
    const uint64_t ad = smem_desc(smem_u32(sA)), bd = smem_desc(smem_u32(sB));
    const uint32_t idesc = instr_desc<MODE>(256, false);
    // commit groups of 256 MMAs alternate between two barriers (a barrier never has two
    // commits outstanding); group g completes phase g / 2 of barrier g % 2
    auto wait_group = [&](int64_t g) {
      return mbar_wait(smem_u32(&bars[g & 1]), (uint32_t)((g >> 1) & 1), abort);
    };
    int64_t groups = 0;
    bool ok = true;
    for (int64_t i0 = 0; i0 < iters && ok; i0 += 16) {   // iters is a multiple of 256
      if (tid == 0) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
          mma<MODE>(tmem + (uint32_t)((u & 1) * 256), ad, bd, idesc, (i0 + u) >= 2 ? 1u : 0u);
      }
      if (((i0 + 15) & 255) == 255) {
        if (tid == 0) mma_commit(smem_u32(&bars[groups & 1]));
        __syncwarp();
        if (groups > 0) ok = wait_group(groups - 1);   // at most two groups in flight
        ++groups;
      }
    }
    if (ok && groups > 0) wait_group(groups - 1);   // the last group covers every MMA
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

template <int MODE>
int run_tc_probe(int64_t iters, double* tflops, cudaStream_t st) {
  auto kern = tc_probe_kernel<MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
  if (e != cudaSuccess) return (int)e;
  const int grid = num_sms();
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return (int)cudaErrorUnknown;
  iters = (iters + 255) / 256 * 256;
  kern<<<grid, 128, kProbeSmem, st>>>((iters / 8 + 255) / 256 * 256);   // warm-up
  cudaEventRecord(e0, st);
  kern<<<grid, 128, kProbeSmem, st>>>(iters);
  cudaEventRecord(e1, st);
  count_launch(2);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  const double flop_per_mma = 2.0 * kRows * 256 * Mode<MODE>::KS;
  *tflops = (double)grid * (double)iters * flop_per_mma / (ms * 1e-3) / 1e12;
  return 0;
}

}  // namespace

bool tc_eligible(int precision, int64_t K, int64_t N, int64_t J, int flags) {
  // default tiles are 128 columns wide (N <= 128 or whole 128-column tiles); fast ones
  // 256 (N <= 256 or whole 256-column tiles)
  const int64_t nt = (flags & kTcFast) ? 256 : 128;
  const bool n_ok = N % 16 == 0 && (N <= nt || N % nt == 0);
  if (precision == QFX_PREC_C3M_BF16X3 || precision == QFX_PREC_C3M_BF16X2)
    return n_ok && K % 16 == 0 && J >= kRows;
  if (precision == QFX_PREC_C3M_TF32X3) return n_ok && K % 8 == 0 && J >= kRows;
  return false;
}

uint64_t tc_scratch_bytes(int precision, int64_t K, int64_t N) {
  // per k-stage and column n: 3 planes per term (the embedded layout of default tiles)
  if (precision == QFX_PREC_C3M_BF16X3) return (uint64_t)(K / 16) * 9 * (uint64_t)N * 32;
  if (precision == QFX_PREC_C3M_BF16X2) return (uint64_t)(K / 16) * 6 * (uint64_t)N * 32;
  if (precision == QFX_PREC_C3M_TF32X3) return (uint64_t)(K / 8) * 6 * (uint64_t)N * 32;
  return 0;
}

int launch_step_tc(const void* S, int64_t s_stride, const void* B, int64_t b_stride, void* C,
                   int64_t c_stride, int64_t P, int64_t K, int64_t N, int64_t NL, int64_t Sd,
                   int batch, int precision, char* scratch, int64_t scratch_stride, void* stream,
                   int flags) {
  cudaStream_t st = (cudaStream_t)stream;
  const int beta = (flags & kTcBeta) ? 1 : 0;
  const bool fast = (flags & kTcFast) != 0;
  const int withhold = (flags & kTcWithhold) ? 1 : 0;
  const bool no_tma = (flags & kTcNoTma) != 0;
  if (precision == QFX_PREC_C3M_BF16X3)
    return fast ? launch_tc_mode<QFX_PREC_C3M_BF16X3, false>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                             Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st)
                : launch_tc_mode<QFX_PREC_C3M_BF16X3, true>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                            Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st);
  if (precision == QFX_PREC_C3M_BF16X2)
    return fast ? launch_tc_mode<QFX_PREC_C3M_BF16X2, false>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                             Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st)
                : launch_tc_mode<QFX_PREC_C3M_BF16X2, true>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                            Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st);
  if (precision == QFX_PREC_C3M_TF32X3)
    return fast ? launch_tc_mode<QFX_PREC_C3M_TF32X3, false>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                             Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st)
                : launch_tc_mode<QFX_PREC_C3M_TF32X3, true>(S, s_stride, B, b_stride, C, c_stride, P, K, N, NL,
                                                            Sd, batch, scratch, scratch_stride, withhold, no_tma, beta, st);
  return (int)cudaErrorInvalidValue;
}

int tc_probe(int precision, int64_t iters, double* tflops, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == QFX_PREC_C3M_BF16X3 || precision == QFX_PREC_C3M_BF16X2)
    return run_tc_probe<QFX_PREC_C3M_BF16X3>(iters, tflops, st);
  if (precision == QFX_PREC_C3M_TF32X3) return run_tc_probe<QFX_PREC_C3M_TF32X3>(iters, tflops, st);
  return (int)cudaErrorInvalidValue;
}

int tc_prepare_attributes() {
  (void)tensor_map_encoder();   // resolve the driver entry point outside any capture
  int e = 0;
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_BF16X3, true>();
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_BF16X3, false>();
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_BF16X2, true>();
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_BF16X2, false>();
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_TF32X3, true>();
  if (!e) e = ensure_tc_attr<QFX_PREC_C3M_TF32X3, false>();
  return e;
}

int tc_take_status() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)) != cudaSuccess) return -1;
  if (v) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_tc_status, &z, sizeof(z));
  }
  return (int)v;
}

}  // namespace qfx
