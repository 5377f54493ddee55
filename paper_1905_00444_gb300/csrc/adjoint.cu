// Adjoint of the amplitude contraction: Wirtinger gradients of a real loss with respect
// to every gate tensor (PyTorch convention: grad = dL/dRe + i dL/dIm = 2 dL/dconj).
//
// The amplitude is multilinear in the site tensors and each gate sits in one site's time
// fold (two sites for a two-qubit gate), so reverse mode is exact:
//   forward   L_{i+1}[nh][p][nl][s] = sum_k S_i[k][nh*NL+nl] L_i[p][k][s]      (Sec. III.E)
//   reverse   R_i[p][k][s]          = sum_n conj(S_i[k][n]) R_{i+1}[nh][p][nl][s]
//             Gbar_{S_i}[k][n]      = sum_{p,s} conj(L_i[p][k][s]) R_{i+1}[nh][p][nl][s]
//   seed      R_n = upstream gradient of the amplitudes (scaled by 2^-m)
//   fold      T[idx] = <x| O_M .. O_1 |0>:  dT/dG[a][b] = w_j[a] u_{j-1}[b] with
//             u_{j-1} = O_{j-1}..O_1|0>, w_j = <x|O_M..O_{j+1}; grad G = sum Gbar_T conj(dT/dG).
//             A general two-qubit gate's q1 event applies the block B_k of its 2-bit leg k:
//             the same formula per element, summed separately for each k, and entry
//             (o1, i1) of B_k (k = 2*o0 + i0) is the gate's G[2*o0 + o1][2*i0 + i1].
// Boundaries: the forward sweep keeps every step's output when they fit the plan's
// adjoint_store_bytes; otherwise it keeps the boundary at the start of every line and the
// reverse sweep recomputes one line's boundaries from its checkpoint before walking it
// backwards ((lines + line length + 2) boundary tensors instead of one per site).
// Scaling: sites were scaled by 2^-e_s and the amplitude by 2^E (E = sum e_s), so the
// gradient of site s is 2^(E - e_s + m) times what the reverse sweep computes; that
// factor is applied in FP64 when the per-event partials are reduced.
// All partial sums are reduced in a fixed order, so results are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int kT = 256;
constexpr int kMaxEvents = 64;     // events per site the fold adjoint supports
constexpr int64_t kGradsBlocks = 304;   // site-gradient grid target: 2 blocks per SM of 152

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }


// ---- seed: R_n[f(o)] = gbar[o] * 2^-m ------------------------------------------------
__global__ void __launch_bounds__(kT) seed_kernel(const double* __restrict__ gout, const int32_t* __restrict__ open_perm,
                                                  int n_open, float2* R, int* m_out) {
  __shared__ double red[kT];
  const int64_t per = int64_t(1) << n_open;
  double mx = 0.0;
  for (int64_t o = threadIdx.x; o < per; o += kT) mx = fmax(mx, fmax(fabs(gout[2 * o]), fabs(gout[2 * o + 1])));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = kT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  int m = 0;
  if (red[0] > 0.0) frexp(red[0], &m);
  if (threadIdx.x == 0) *m_out = m;
  for (int64_t o = threadIdx.x; o < per; o += kT) {
    int64_t f = 0;
    for (int i = 0; i < n_open; ++i) f |= ((o >> i) & 1) << open_perm[i];
    R[f] = make_float2((float)ldexp(gout[2 * o], -m), (float)ldexp(gout[2 * o + 1], -m));
  }
}

// ---- reverse step: Rout[p][k][s] = sum_n conj(S[k][n]) Rin[n/NL][p][n%NL][s] ------------
// BM (16 or 64) rows k by 64 columns j per block; thread (ty, tx) owns BM/16 x 4 outputs.
template <int BM>
__global__ void __launch_bounds__(kT) rstep_kernel(const float2* __restrict__ S, const float2* __restrict__ Rin,
                                                   float2* __restrict__ Rout, int64_t P, int64_t K,
                                                   int64_t N, int64_t NL, int64_t Sd) {
  constexpr int BJ = 64, BR = 16, TMK = BM / 16;
  static_assert(kT == 256 && (BM == 16 || BM == 64), "thread layout");
  __shared__ float2 As[BR][BM + 1];
  __shared__ float2 Bs[BR][BJ + 1];
  const int64_t J = P * Sd, KT_ = (K + BM - 1) / BM;
  const int64_t kt = blockIdx.x % KT_, jt = blockIdx.x / KT_;
  const int64_t k0 = kt * BM, j0 = jt * BJ;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t strideNH = P * NL * Sd;
  // B elements of this thread: column c = threadIdx.x % BJ, rows r0 + 4 i; the j part of
  // the address is computed once, the n part with 32-bit divisions
  const int c = threadIdx.x % BJ, r0 = threadIdx.x / BJ;
  const int64_t jc = j0 + c;
  const bool jok = jc < J;
  const int64_t joff = jok ? (jc / Sd) * NL * Sd + jc % Sd : 0;
  const int NLi = (int)NL;
  float2 acc[TMK][4];
#pragma unroll
  for (int i = 0; i < TMK; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int64_t n0 = 0; n0 < N; n0 += BR) {
#pragma unroll
    for (int i = 0; i < TMK; ++i) {   // A: BR x BM elements, BM / 16 per thread
      const int e = threadIdx.x + i * kT;
      const int ra = e / BM, ca = e % BM;
      const int64_t k = k0 + ca, n = n0 + ra;
      float2 v = make_float2(0.f, 0.f);
      if (k < K && n < N) { v = S[k * N + n]; v.y = -v.y; }
      As[ra][ca] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {     // B: BR x BJ elements, 4 per thread
      const int r = r0 + i * (kT / BJ);
      const int64_t n = n0 + r;
      float2 b = make_float2(0.f, 0.f);
      if (jok && n < N) {
        const int ni = (int)n;
        b = Rin[(int64_t)(ni / NLi) * strideNH + (int64_t)(ni % NLi) * Sd + joff];
      }
      Bs[r][c] = b;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      float2 a[TMK], b[4];
#pragma unroll
      for (int i = 0; i < TMK; ++i) a[i] = As[r][ty * TMK + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[r][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < TMK; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t jj = j0 + tx * 4 + j;
    if (jj >= J) continue;
    const int64_t jp = jj / Sd, js = jj - jp * Sd;
#pragma unroll
    for (int i = 0; i < TMK; ++i) {
      const int64_t k = k0 + ty * TMK + i;
      if (k < K) Rout[jp * K * Sd + k * Sd + js] = acc[i][j];
    }
  }
}

// ---- conjugate transposes of the site matrices for the reverse steps with NL = N -------
// Such a reverse step is a forward step of the step tile: Rout[p][k][s] =
// sum_n S'[n][k] Rin[p][n][s] with S'[n][k] = conj(S[k][n]) (K and N swapped, NL = K).
// One launch for all of them: entry y of the table below transposes its K x N matrix in
// 32 x 32 tiles through shared memory (tile x of ceil(K/32) * ceil(N/32); extra blocks exit).
constexpr int kConjMax = 144;
struct ConjTable {
  int64_t off[kConjMax];   // element offset of the site matrix (and of its transpose)
  int32_t K[kConjMax], N[kConjMax];
  int32_t count;
};
__global__ void __launch_bounds__(kT) conj_transpose_kernel(const float2* __restrict__ sites,
                                                            float2* __restrict__ sconj, const ConjTable tab) {
  __shared__ float2 tile[32][33];
  const int y = blockIdx.y;
  const int64_t K = tab.K[y], N = tab.N[y];
  const int64_t tk = (K + 31) / 32, tn = (N + 31) / 32;
  if ((int64_t)blockIdx.x >= tk * tn) return;   // block-uniform
  const int64_t k0 = (blockIdx.x % tk) * 32, n0 = (blockIdx.x / tk) * 32;
  const float2* S = sites + tab.off[y];
  float2* St = sconj + tab.off[y];
  const int x = threadIdx.x & 31, r = threadIdx.x >> 5;
  for (int rr = r; rr < 32; rr += kT / 32) {   // read rows k, columns n (coalesced along n)
    const int64_t k = k0 + rr, n = n0 + x;
    if (k < K && n < N) tile[rr][x] = S[k * N + n];
  }
  __syncthreads();
  for (int rr = r; rr < 32; rr += kT / 32) {   // write rows n, columns k (coalesced along k)
    const int64_t n = n0 + rr, k = k0 + x;
    if (k < K && n < N) {
      const float2 v = tile[x][rr];
      St[n * K + k] = make_float2(v.x, -v.y);
    }
  }
}

int launch_rstep(const float2* S, const float2* Rin, float2* Rout, int64_t P, int64_t K, int64_t N, int64_t NL,
                 int64_t Sd, cudaStream_t st) {
  const int64_t J = P * Sd;
  if (K <= 16) {
    const int64_t blocks = ((K + 15) / 16) * ((J + 63) / 64);
    rstep_kernel<16><<<(unsigned)blocks, kT, 0, st>>>(S, Rin, Rout, P, K, N, NL, Sd);
  } else {
    const int64_t blocks = ((K + 63) / 64) * ((J + 63) / 64);
    rstep_kernel<64><<<(unsigned)blocks, kT, 0, st>>>(S, Rin, Rout, P, K, N, NL, Sd);
  }
  return (int)cudaGetLastError();
}

// ---- site gradient, split over columns: part[c][k][n] = sum_{j in c} conj(L(k,j)) R(n,j) ----
// BM x BN output tiles (16 or 64 each, so that K or N of 8 or 16 does not fill 64-wide
// tiles with zeros); thread (ty, tx) owns BM/16 x BN/16 outputs.  The columns j are cut
// into chunks so that the grid has about kGradsBlocks blocks whatever K and N are.  Slabs
// of 16 columns of L and R move through two shared-memory buffers by cp.async (the next
// slab's copies overlap this one's FMAs); a thread's column j steps through (p, s) without
// divisions.
__device__ __forceinline__ void g_cp_async8(void* smem, const void* gmem, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 8 : 0));
}
template <int BM, int BN>
__global__ void __launch_bounds__(kT) grads_kernel(const float2* __restrict__ Lin, const float2* __restrict__ Rin,
                                                   float2* __restrict__ part, int64_t P, int64_t K,
                                                   int64_t N, int64_t NL, int64_t Sd, int64_t chunk) {
  constexpr int BJ = 16, TMK = BM / 16, TNN = BN / 16;
  constexpr int LA = BM + 2, LB = BN + 2;   // rows of 16-byte multiples, 2-way store conflicts
  static_assert(kT == 256 && BM % 16 == 0 && BN % 16 == 0, "thread layout");
  __shared__ __align__(16) float2 As[2][BJ][LA];
  __shared__ __align__(16) float2 Bs[2][BJ][LB];
  const int64_t J = P * Sd;
  const int64_t k0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t jb = (int64_t)blockIdx.z * chunk, je = min(J, jb + chunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t strideNH = P * NL * Sd;
  // every element this thread copies has column jj = threadIdx.x % BJ of the slab and rows
  // c0 + 16 i: the k and n parts of the addresses are fixed
  const int jj = threadIdx.x % BJ, c0 = threadIdx.x / BJ;
  int64_t koff[TMK], noff[TNN];
#pragma unroll
  for (int i = 0; i < TMK; ++i) {
    const int64_t k = k0 + c0 + 16 * i;
    koff[i] = k < K ? k * Sd : -1;
  }
#pragma unroll
  for (int i = 0; i < TNN; ++i) {
    const int64_t n = n0 + c0 + 16 * i;
    noff[i] = n < N ? (n / NL) * strideNH + (n % NL) * Sd : -1;
  }
  int64_t j = jb + jj;
  int64_t jp = j / Sd, js = j - jp * Sd;
  auto load = [&](int buf) {
    const bool jok = j < je;
    const float2* Lp = Lin + jp * K * Sd + js;
    const float2* Rp = Rin + jp * NL * Sd + js;
#pragma unroll
    for (int i = 0; i < TMK; ++i) {
      const bool ok = jok && koff[i] >= 0;
      g_cp_async8(&As[buf][jj][c0 + 16 * i], ok ? Lp + koff[i] : Lin, ok);
    }
#pragma unroll
    for (int i = 0; i < TNN; ++i) {
      const bool ok = jok && noff[i] >= 0;
      g_cp_async8(&Bs[buf][jj][c0 + 16 * i], ok ? Rp + noff[i] : Rin, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    j += BJ;   // this thread's column in the next slab
    js += BJ;
    while (js >= Sd) { js -= Sd; ++jp; }
  };
  float2 acc[TMK][TNN];
#pragma unroll
  for (int i = 0; i < TMK; ++i)
#pragma unroll
    for (int q = 0; q < TNN; ++q) acc[i][q] = make_float2(0.f, 0.f);
  const int64_t nslab = (je - jb + BJ - 1) / BJ;
  if (nslab > 0) load(0);
  for (int64_t t = 0; t < nslab; ++t) {
    const int buf = (int)(t & 1);
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();   // slab t landed for every thread; slab t-1's buffer is free
    if (t + 1 < nslab) load(buf ^ 1);
#pragma unroll
    for (int r = 0; r < BJ; ++r) {
      float2 a[TMK], b[TNN];
      if constexpr (TMK % 2 == 0) {   // 16-byte pairs (ty * TMK even, rows 16-byte multiples)
#pragma unroll
        for (int i = 0; i < TMK; i += 2) {
          const float4 v = *reinterpret_cast<const float4*>(&As[buf][r][ty * TMK + i]);
          a[i] = make_float2(v.x, v.y);
          a[i + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < TMK; ++i) a[i] = As[buf][r][ty * TMK + i];
      }
      if constexpr (TNN % 2 == 0) {
#pragma unroll
        for (int q = 0; q < TNN; q += 2) {
          const float4 v = *reinterpret_cast<const float4*>(&Bs[buf][r][tx * TNN + q]);
          b[q] = make_float2(v.x, v.y);
          b[q + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int q = 0; q < TNN; ++q) b[q] = Bs[buf][r][tx * TNN + q];
      }
#pragma unroll
      for (int i = 0; i < TMK; ++i)
#pragma unroll
        for (int q = 0; q < TNN; ++q) {   // conj(a) * b
          acc[i][q].x = fmaf(a[i].x, b[q].x, fmaf(a[i].y, b[q].y, acc[i][q].x));
          acc[i][q].y = fmaf(a[i].x, b[q].y, fmaf(-a[i].y, b[q].x, acc[i][q].y));
        }
    }
  }
  float2* out = part + (int64_t)blockIdx.z * K * N;
#pragma unroll
  for (int i = 0; i < TMK; ++i)
#pragma unroll
    for (int q = 0; q < TNN; ++q) {
      const int64_t k = k0 + ty * TMK + i, n = n0 + tx * TNN + q;
      if (k < K && n < N) out[k * N + n] = acc[i][q];
    }
}

// Geometry of the site-gradient GEMM of one step (the same on the host for the workspace
// size and for the launch).
struct GradsGeom {
  int bm, bn;
  int64_t chunk, chunks;
};
GradsGeom grads_geom(int64_t K, int64_t N, int64_t J) {
  GradsGeom g;
  g.bm = K <= 16 ? 16 : 64;
  g.bn = N <= 16 ? 16 : 64;
  const int64_t tiles = ((K + g.bm - 1) / g.bm) * ((N + g.bn - 1) / g.bn);
  const int64_t steps = (J + 15) / 16;
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>(steps, (kGradsBlocks + tiles - 1) / tiles));
  g.chunk = ((steps + want - 1) / want) * 16;
  g.chunks = (J + g.chunk - 1) / g.chunk;
  return g;
}

int launch_grads(const GradsGeom& g, const float2* Lin, const float2* Rin, float2* part, int64_t P, int64_t K,
                 int64_t N, int64_t NL, int64_t Sd, cudaStream_t st) {
  dim3 grid((unsigned)((K + g.bm - 1) / g.bm), (unsigned)((N + g.bn - 1) / g.bn), (unsigned)g.chunks);
  if (g.bm == 16 && g.bn == 16) grads_kernel<16, 16><<<grid, kT, 0, st>>>(Lin, Rin, part, P, K, N, NL, Sd, g.chunk);
  else if (g.bm == 16) grads_kernel<16, 64><<<grid, kT, 0, st>>>(Lin, Rin, part, P, K, N, NL, Sd, g.chunk);
  else if (g.bn == 16) grads_kernel<64, 16><<<grid, kT, 0, st>>>(Lin, Rin, part, P, K, N, NL, Sd, g.chunk);
  else grads_kernel<64, 64><<<grid, kT, 0, st>>>(Lin, Rin, part, P, K, N, NL, Sd, g.chunk);
  return (int)cudaGetLastError();
}

// One warp per output element: lane l sums chunks l, l + 32, ... in order, then a fixed
// butterfly adds the lanes (deterministic).
__global__ void __launch_bounds__(kT) reduce_chunks_kernel(const float2* __restrict__ part, int64_t chunks,
                                                           int64_t KN, float2* __restrict__ out) {
  const int64_t t = ((int64_t)blockIdx.x * kT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= KN) return;   // warp-uniform: t is the same for all lanes of a warp
  float re = 0.f, im = 0.f;
  for (int64_t c = lane; c < chunks; c += 32) {
    const float2 v = part[c * KN + t];
    re += v.x;
    im += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) out[t] = make_float2(re, im);
}

// ---- fold adjoint: per-block partial gradients of every event's matrix ----------------
// One thread per site-tensor element.  The per-element chains and the warp sums run in
// FP32: the site gradient they consume is FP32 already, and nev FP32 roundings (relative
// nev * 2^-24) stay far below its error, while this GPU's FP64 rate is 1/64 of FP32.  The
// warp sums leave the registers as FP64 and every later sum is FP64.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {   // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// complex entry i of a gate matrix in the fold's float-float table (16 floats per matrix,
// a (hi, lo) pair per FP64 real): its FP32 value is the hi parts, the round-to-nearest of
// the FP64 entries, read without a conversion from FP64
__device__ __forceinline__ float2 mat_entry(const float* m, int i) {
  return make_float2(m[4 * i], m[4 * i + 2]);
}

// Sums v[0..7] over the warp by halving: after the exchanges at distance 16, 8 and 4 each
// lane holds one entry, e = 4 * bit4 + 2 * bit3 + bit2 of its lane index, summed over the
// lanes that differ in those bits; distances 2 and 1 finish it (9 shuffles instead of 40).
__device__ __forceinline__ float warp_sum8(float v[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float send = h16 ? v[t] : v[t + 4];
    const float keep = h16 ? v[t + 4] : v[t];
    v[t] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float send = h8 ? v[t] : v[t + 2];
    const float keep = h8 ? v[t + 2] : v[t];
    v[t] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const float send = h4 ? v[0] : v[1];
    const float keep = h4 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float x = v[0];
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

// Partial slots of an event: a general gate's q1 block B_k has 4 x 4 entries, one set of 4
// per leg value k (each element sees one k); every other event has one set of 4 (zero for
// parameter-free events).  kMaxEvents bounds a site's slots.
__host__ __device__ __forceinline__ int ev_slots(int kind) { return kind == EV_BLOCK ? 4 : 1; }

__global__ void __launch_bounds__(kT) fold_backward_kernel(
    const FoldSite* __restrict__ sites, const FoldEvent* __restrict__ events, const float* __restrict__ matsf,
    const CutDev* __restrict__ cuts, int n_cuts, const uint64_t* __restrict__ x1w, int64_t sid,
    const float2* __restrict__ sgrad, double* __restrict__ bpart, const int64_t* __restrict__ part_off) {
  __shared__ double wpart[kT / 32][kMaxEvents][8];
  const FoldSite st = sites[blockIdx.y];
  const int nev = st.ev_end - st.ev_begin;
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if ((int64_t)blockIdx.x * kT >= st.size) return;   // block-uniform
  const bool active = i < st.size;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t off[4] = {0, 0, 0, 0};
  for (int c = 0; c < n_cuts; ++c) {
    const CutDev cd = cuts[c];
    const int64_t digit = (sid / cd.suffix) % cd.radix;
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (st.edge[s] == cd.edge) off[s] = digit * cd.size;
  }
  int64_t r = active ? i : 0;
  const int64_t vd = r % st.dim[4]; r /= st.dim[4];
  const int64_t vr = r % st.dim[3]; r /= st.dim[3];
  const int64_t vx = r % st.dim[2]; r /= st.dim[2];
  const int64_t vl = r % st.dim[1]; r /= st.dim[1];
  const int64_t vu = r;
  const uint64_t val0 = (uint64_t)(vu + off[0]), val1 = (uint64_t)(vl + off[1]);
  const uint64_t val2 = (uint64_t)(vr + off[2]), val3 = (uint64_t)(vd + off[3]);
  const int xv = st.x_open ? (int)vx : (int)((x1w[st.qubit >> 6] >> (st.qubit & 63)) & 1ull);
  const float2 zero = make_float2(0.f, 0.f);
  auto leg = [&](const FoldEvent& ev, uint64_t width_mask) {
    const uint64_t bv = ev.slot == 0 ? val0 : ev.slot == 1 ? val1 : ev.slot == 2 ? val2 : val3;
    return (int)((bv >> ev.bit) & width_mask);
  };
  // forward: states u_j before each event
  float2 u0[kMaxEvents + 1], u1[kMaxEvents + 1];
  u0[0] = make_float2(1.f, 0.f);
  u1[0] = zero;
  int n_slots = 0;
  for (int j = 0; j < nev; ++j) {
    const FoldEvent ev = events[st.ev_begin + j];
    n_slots += ev_slots(ev.kind);
    const float* m = matsf + 16 * (int64_t)ev.mat;
    float2 a = u0[j], c = u1[j];
    if (ev.kind == EV_GATE || ev.kind == EV_BLOCK) {
      const float* g = ev.kind == EV_GATE ? m : m + 16 * leg(ev, 3);
      const float2 g00 = mat_entry(g, 0), g01 = mat_entry(g, 1), g10 = mat_entry(g, 2), g11 = mat_entry(g, 3);
      const float2 p0 = cmulf(g00, a), q0 = cmulf(g01, c), p1 = cmulf(g10, a), q1 = cmulf(g11, c);
      a = make_float2(p0.x + q0.x, p0.y + q0.y);
      c = make_float2(p1.x + q1.x, p1.y + q1.y);
    } else if (ev.kind == EV_ELEM) {                 // |o0><i0|, k = 2*o0 + i0
      const int k = leg(ev, 3);
      const float2 src = (k & 1) ? c : a;
      a = (k >> 1) ? zero : src;
      c = (k >> 1) ? src : zero;
    } else {
      const int k = leg(ev, 1);
      if (ev.kind == EV_PROJ) {
        if (k) a = zero;
        else   c = zero;
      } else {
        a = cmulf(a, mat_entry(m, 2 * k));
        c = cmulf(c, mat_entry(m, 2 * k + 1));
      }
    }
    u0[j + 1] = a;
    u1[j + 1] = c;
  }
  const float2 g = active ? sgrad[st.offset + i] : zero;
  // backward: row vector w = <x| O_M .. O_{j+1}
  float2 w0 = make_float2(xv == 0 ? 1.f : 0.f, 0.f), w1 = make_float2(xv == 1 ? 1.f : 0.f, 0.f);
  int sl = n_slots;
  for (int j = nev - 1; j >= 0; --j) {
    const FoldEvent ev = events[st.ev_begin + j];
    const float* m = matsf + 16 * (int64_t)ev.mat;
    const float2 a = u0[j], c = u1[j];
    sl -= ev_slots(ev.kind);
    const int k = ev.kind == EV_GATE ? 0 : leg(ev, (ev.kind == EV_ELEM || ev.kind == EV_BLOCK) ? 3 : 1);
    float2 d[4] = {zero, zero, zero, zero};
    if (ev.kind == EV_GATE || ev.kind == EV_BLOCK) {
      d[0] = cmulcf(g, cmulf(w0, a));   // dG[0][0] = w0 u0
      d[1] = cmulcf(g, cmulf(w0, c));   // dG[0][1] = w0 u1
      d[2] = cmulcf(g, cmulf(w1, a));   // dG[1][0] = w1 u0
      d[3] = cmulcf(g, cmulf(w1, c));   // dG[1][1] = w1 u1
    } else if (ev.kind == EV_DIAG) {
      d[2 * k + 0] = cmulcf(g, cmulf(w0, a));
      d[2 * k + 1] = cmulcf(g, cmulf(w1, c));
    }
    // event-uniform branches: projections and elementary matrices have no entries
    if (ev.kind == EV_PROJ || ev.kind == EV_ELEM) {
      if (lane < 8) wpart[warp][sl][lane] = 0.0;
    } else {
      for (int kk = 0; kk < ev_slots(ev.kind); ++kk) {   // a block's sum goes to its k's slot
        const bool mine = ev.kind != EV_BLOCK || kk == k;
        float v[8] = {mine ? d[0].x : 0.f, mine ? d[0].y : 0.f, mine ? d[1].x : 0.f, mine ? d[1].y : 0.f,
                      mine ? d[2].x : 0.f, mine ? d[2].y : 0.f, mine ? d[3].x : 0.f, mine ? d[3].y : 0.f};
        const float sum = warp_sum8(v, lane);
        if ((lane & 3) == 0)
          wpart[warp][sl + kk][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = sum;
      }
    }
    // w <- w O_j
    if (ev.kind == EV_GATE || ev.kind == EV_BLOCK) {
      const float* gm = ev.kind == EV_GATE ? m : m + 16 * k;
      const float2 g00 = mat_entry(gm, 0), g01 = mat_entry(gm, 1), g10 = mat_entry(gm, 2), g11 = mat_entry(gm, 3);
      const float2 p0 = cmulf(w0, g00), q0 = cmulf(w1, g10), p1 = cmulf(w0, g01), q1 = cmulf(w1, g11);
      w0 = make_float2(p0.x + q0.x, p0.y + q0.y);
      w1 = make_float2(p1.x + q1.x, p1.y + q1.y);
    } else if (ev.kind == EV_ELEM) {                 // (w |o0><i0|)[col] = w[o0] delta(col, i0)
      const float2 src = (k >> 1) ? w1 : w0;
      w0 = (k & 1) ? zero : src;
      w1 = (k & 1) ? src : zero;
    } else if (ev.kind == EV_PROJ) {
      if (k) w0 = zero;
      else   w1 = zero;
    } else {
      w0 = cmulf(w0, mat_entry(m, 2 * k));
      w1 = cmulf(w1, mat_entry(m, 2 * k + 1));
    }
  }
  __syncthreads();
  double* outp = bpart + part_off[blockIdx.y] + (int64_t)blockIdx.x * n_slots * 8;
  for (int t = threadIdx.x; t < n_slots * 8; t += kT) {
    const int j = t / 8, e = t % 8;
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += wpart[w][j][e];
    outp[j * 8 + e] = s;
  }
}

// one thread per (event, double of its up to 4 slots): sum the site's blocks, apply
// 2^(E - e_s + m); evgrad holds 32 doubles per event
__global__ void __launch_bounds__(kT) event_reduce_kernel(const FoldSite* __restrict__ sites, int n_sites,
                                                          const FoldEvent* __restrict__ events,
                                                          const double* __restrict__ bpart,
                                                          const int64_t* __restrict__ part_off,
                                                          const int* __restrict__ hdr_exps, const int* m_ptr,
                                                          int n_events, double* __restrict__ evgrad) {
  const int t = blockIdx.x * kT + threadIdx.x;
  if (t >= n_events * 32) return;
  const int e = t / 32, entry = t % 32;
  int s = 0;
  for (int q = 0; q < n_sites; ++q)
    if (e >= sites[q].ev_begin && e < sites[q].ev_end) s = q;
  const FoldSite st = sites[s];
  int slot = 0, n_slots = 0;
  for (int j = st.ev_begin; j < st.ev_end; ++j) {
    if (j == e) slot = n_slots;
    n_slots += ev_slots(events[j].kind);
  }
  if (entry >= 8 * ev_slots(events[e].kind)) {
    evgrad[t] = 0.0;
    return;
  }
  const int64_t nblk = (st.size + kT - 1) / kT;
  double sum = 0.0;
  for (int64_t bk = 0; bk < nblk; ++bk) sum += bpart[part_off[s] + bk * n_slots * 8 + slot * 8 + entry];
  int E = 0;
  for (int q = 0; q < n_sites; ++q) E += hdr_exps[q];
  evgrad[t] = ldexp(sum, E - hdr_exps[s] + *m_ptr);
}

// one thread per (gate, double of its `per_gate` complex entries): add the gate's events
// into the output (item order).  A general gate's entry G[r][c] is entry (o1, i1) of the
// block B_k of its q1 event, k = 2*o0 + i0 (r = 2*o0 + o1, c = 2*i0 + i1); other gates
// fill their first 4 entries.
__global__ void __launch_bounds__(kT) gate_accum_kernel(const int32_t* __restrict__ gate_ev,
                                                        const FoldEvent* __restrict__ events, int n_gates,
                                                        int per_gate, const double* __restrict__ evgrad,
                                                        double* grad) {
  const int t = blockIdx.x * kT + threadIdx.x;
  if (t >= n_gates * 2 * per_gate) return;
  const int gte = t / (2 * per_gate), ent = t % (2 * per_gate), ce = ent / 2, ri = ent & 1;
  int block = -1;
  for (int q = 0; q < 2; ++q) {
    const int e = gate_ev[2 * gte + q];
    if (e >= 0 && events[e].kind == EV_BLOCK) block = e;
  }
  double s = 0.0;
  if (block >= 0) {
    const int r = ce / 4, c = ce % 4;
    const int k = 2 * (r >> 1) + (c >> 1), bi = 2 * (r & 1) + (c & 1);
    s = evgrad[block * 32 + (k * 4 + bi) * 2 + ri];
  } else if (ce < 4) {
    for (int q = 0; q < 2; ++q) {
      const int e = gate_ev[2 * gte + q];
      if (e >= 0) s += evgrad[e * 32 + ce * 2 + ri];
    }
  }
  grad[t] += s;
}

struct BwdLayout {
  uint64_t tab, hdr, sites, sconj, sgrad, ckpt, lb, rr, gpart, bpart, evgrad, total;
};

// Every step output is kept (no recomputation in the reverse sweep) when all of them fit in
// the plan's adjoint_store_bytes; larger plans keep one checkpoint per line and recompute it.
bool full_store(const qfx_plan* p) {
  return (uint64_t)p->n * a256((uint64_t)p->max_elements * 8) <= p->adjoint_store_bytes;
}

int64_t site_slots(const qfx_plan* p, const FoldSite& fs) {
  int64_t n = 0;
  for (int j = fs.ev_begin; j < fs.ev_end; ++j) n += ev_slots(p->events[j].kind);
  return n;
}

BwdLayout bwd_layout(const qfx_plan* p) {
  BwdLayout L{};
  const uint64_t B = a256((uint64_t)p->max_elements * 8);
  uint64_t o = 0;
  L.tab = o; o += table_bytes(p);   // the plan's tables, copied in by every call
  L.hdr = o; o += a256((uint64_t)p->n * 8 + 16);
  L.sites = o; o += a256((uint64_t)p->site_total * 8);
  L.sconj = o; o += a256((uint64_t)p->site_total * 8);
  L.sgrad = o; o += a256((uint64_t)p->site_total * 8);
  if (full_store(p)) {   // ckpt holds the output of every step
    L.ckpt = o; o += (uint64_t)p->n * B;
    L.lb = L.ckpt;
  } else {
    L.ckpt = o; o += (uint64_t)p->lines * B;
    L.lb = o; o += (uint64_t)p->line_len * B;
  }
  L.rr = o; o += 2 * B;
  uint64_t gp = 0;
  for (size_t i = 1; i < p->steps.size(); ++i) {
    const Step& s = p->steps[i];
    const GradsGeom g = grads_geom(s.K, s.N, s.P * s.Sd);
    gp = std::max(gp, (uint64_t)g.chunks * (uint64_t)s.K * (uint64_t)s.N * 8);
  }
  L.gpart = o; o += a256(gp);
  uint64_t bp = 0;
  for (const auto& fs : p->sites) bp += (uint64_t)((fs.size + kT - 1) / kT) * site_slots(p, fs) * 8;
  L.bpart = o; o += a256(bp * 8);
  L.evgrad = o; o += a256((uint64_t)p->events.size() * 32 * 8);
  L.total = o;
  return L;
}

}  // namespace

// Fold-adjoint partials of one site: one slot per event slot for each 256-element block.
int64_t adjoint_site_partials(const qfx_plan* p, const FoldSite& fs) {
  return ((fs.size + kT - 1) / kT) * site_slots(p, fs) * 8;
}

}  // namespace qfx

using namespace qfx;

extern "C" uint64_t qfx_backward_workspace_bytes(const qfx_plan* p) {
  if (!p) return 0;
  return bwd_layout(p).total;
}

namespace {

qfx_status backward(const qfx_plan* p, const uint64_t* x1, int64_t n_batch, int64_t slice_begin,
                    int64_t slice_end, const double* grad_out, double* grad_gates, int per_gate,
                    void* workspace, size_t ws_bytes, void* stream) {
  if (p && per_gate == 4)
    for (const auto& ev : p->events)
      if (ev.kind == EV_ELEM || ev.kind == EV_BLOCK)
        return fail(QFX_EUNSUPPORTED, "qfx_amplitudes_backward: general (U4) two-qubit gates have 16 "
                                      "entries, more than the 4 per gate of grad_gates "
                                      "(qfx_amplitudes_backward_full writes 16)");
  qfx_status s = check_amplitudes_args(p, x1, n_batch, slice_begin, slice_end, grad_out);
  if (s != QFX_OK) return s;
  if (p->family != 0)
    return fail(QFX_EUNSUPPORTED, "qfx_amplitudes_backward: line-sweep plans only (plan_family 0)");
  if (!grad_gates || !workspace) return fail(QFX_EINVAL, "qfx_amplitudes_backward: NULL argument");
  if (((uintptr_t)workspace & 255) || ((uintptr_t)grad_gates & 15))
    return fail(QFX_EINVAL, "qfx_amplitudes_backward: misaligned workspace or grad_gates");
  for (const auto& fs : p->sites)
    if (site_slots(p, fs) > kMaxEvents)
      return fail(QFX_EUNSUPPORTED, "qfx_amplitudes_backward: a site has more than 64 time-line event "
                                    "slots (a general gate's block takes 4)");
  const BwdLayout Lw = bwd_layout(p);
  if (ws_bytes < Lw.total) return fail(QFX_ENOMEM, "qfx_amplitudes_backward: workspace smaller than qfx_backward_workspace_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  DeviceTables t;
  s = stage_tables(p, ws + Lw.tab, stream, &t);
  if (s != QFX_OK) return s;
  const uint64_t B = a256((uint64_t)p->max_elements * 8);
  const int n = p->n, L = p->line_len, W = p->lines;
  const bool full = full_store(p);
  const int n_open = (int)p->open_sites.size();
  const int64_t per = int64_t(1) << n_open;
  int64_t max_site = 1;
  for (const auto& fs : p->sites) max_site = std::max(max_site, fs.size);
  cudaError_t e;
  e = cudaMemsetAsync(grad_gates, 0, (size_t)p->n_gates * 2 * per_gate * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes_backward: clearing grad_gates");

  char* hdr = ws + Lw.hdr;
  int* exps = (int*)hdr + n;
  int* m_ptr = (int*)(hdr + (uint64_t)n * 8);
  char* sites = ws + Lw.sites;
  float2* sgrad = (float2*)(ws + Lw.sgrad);
  auto ckpt = [&](int w) { return ws + Lw.ckpt + (uint64_t)w * B; };
  auto lb = [&](int j) { return ws + Lw.lb + (uint64_t)j * B; };
  auto rr = [&](int j) { return ws + Lw.rr + (uint64_t)j * B; };
  auto site_ptr = [&](int q) { return sites + (uint64_t)p->sites[q].offset * 8; };
  const int64_t n_items = (slice_end - slice_begin) * n_batch;
  auto step_fwd = [&](int i, const char* in, char* out) -> int {
    const Step& sp = p->steps[i];
    const int v = fill_variant(pick_variant(sp.N, sp.Sd), sp.N, sp.P * sp.Sd, 1);
    return launch_step(site_ptr(sp.site), 0, in, 0, out, 0, sp.P, sp.K, sp.N, sp.NL, sp.Sd, 1, v,
                       QFX_PREC_FP32_SIMT, st);
  };

  // reverse steps with NL = N run on the step tile with the conjugate transpose of their
  // site matrix (conj_transpose_kernel, once per item); the others on rstep_kernel
  ConjTable ctab{};
  std::vector<char> use_conj(p->steps.size(), 0);
  int64_t conj_tiles = 0;
  for (size_t i = 1; i < p->steps.size() && ctab.count < kConjMax; ++i) {
    const Step& sp = p->steps[i];
    const FoldSite& fs = p->sites[sp.site];
    if (sp.NL != sp.N || fs.size != sp.K * sp.N || sp.K > 0x7fffffff || sp.N > 0x7fffffff) continue;
    use_conj[i] = 1;
    ctab.off[ctab.count] = fs.offset;
    ctab.K[ctab.count] = (int32_t)sp.K;
    ctab.N[ctab.count] = (int32_t)sp.N;
    ++ctab.count;
    conj_tiles = std::max(conj_tiles, ((sp.K + 31) / 32) * ((sp.N + 31) / 32));
  }
  float2* sconj = (float2*)(ws + Lw.sconj);

  for (int64_t item = 0; item < n_items; ++item) {
    const int64_t b = item % n_batch, sid = slice_begin + item / n_batch;
    e = cudaMemsetAsync(hdr, 0, (size_t)n * 8 + 16, st);
    if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes_backward: header");
    int err = launch_fold(t, n, max_site, (int)p->cut_dev.size(), x1, p->x1_words, n_batch, slice_begin,
                          item, 1, hdr, 0, sites, 0, 0, st);
    if (!err) err = launch_scale(t, n, max_site, 1, hdr, 0, sites, 0, 0, st);
    if (err) return cuda_fail(err, "qfx_amplitudes_backward: fold");
    if (ctab.count > 0) {
      conj_transpose_kernel<<<dim3((unsigned)conj_tiles, (unsigned)ctab.count), kT, 0, st>>>(
          (const float2*)sites, sconj, ctab);
      count_launch();
    }
    // forward sweep, keeping every step's output (full) or the boundary at the start of
    // every line
    const char* cur = site_ptr(p->steps[0].site);
    int pp = 0;
    for (int i = 1; i < n - 1; ++i) {
      char* out = full ? ckpt(i) : ((i + 1) % L == 0) ? ckpt((i + 1) / L) : rr(pp);
      if (!full && out == rr(pp)) pp ^= 1;
      err = step_fwd(i, cur, out);
      if (err) return cuda_fail(err, "qfx_amplitudes_backward: forward step");
      cur = out;
    }
    // seed from this batch row's upstream gradient
    float2* Rcur = (float2*)rr(0);
    int rsel = 0;
    seed_kernel<<<1, kT, 0, st>>>(grad_out + 2 * b * per, t.open_perm, n_open, Rcur, m_ptr);
    count_launch();
    // reverse: gradient of step i's site from its input Lin and the incoming R, then R
    // through the step
    auto reverse_step = [&](int i, const char* Lin_raw) -> qfx_status {
      const Step& sp = p->steps[i];
      float2* gdst = sgrad + p->sites[sp.site].offset;
      if (i == 0) {
        cudaError_t e2 = cudaMemcpyAsync(gdst, Rcur, (size_t)sp.N * 8, cudaMemcpyDeviceToDevice, st);
        if (e2 != cudaSuccess) return cuda_fail(e2, "qfx_amplitudes_backward: site 0 gradient");
        return QFX_OK;
      }
      const float2* Lin = (const float2*)Lin_raw;
      const int64_t J = sp.P * sp.Sd;
      const GradsGeom gg = grads_geom(sp.K, sp.N, J);
      float2* part = (float2*)(ws + Lw.gpart);
      launch_grads(gg, Lin, Rcur, part, sp.P, sp.K, sp.N, sp.NL, sp.Sd, st);
      const int64_t KN = sp.K * sp.N;
      reduce_chunks_kernel<<<(unsigned)((KN * 32 + kT - 1) / kT), kT, 0, st>>>(part, gg.chunks, KN, gdst);
      float2* Rnext = (float2*)rr(rsel ^ 1);
      if (use_conj[i]) {
        const int v = fill_variant(pick_variant(sp.K, sp.Sd), sp.K, J, 1);
        const int err2 = launch_step(sconj + p->sites[sp.site].offset, 0, Rcur, 0, Rnext, 0, sp.P, sp.N, sp.K,
                                     sp.K, sp.Sd, 1, v, QFX_PREC_FP32_SIMT, st);
        if (err2) return cuda_fail(err2, "qfx_amplitudes_backward: reverse step");
        count_launch(2);
      } else {
        launch_rstep((const float2*)site_ptr(sp.site), Rcur, Rnext, sp.P, sp.K, sp.N, sp.NL, sp.Sd, st);
        count_launch(3);
      }
      rsel ^= 1;
      Rcur = Rnext;
      cudaError_t e2 = cudaGetLastError();
      if (e2 != cudaSuccess) return cuda_fail(e2, "qfx_amplitudes_backward: reverse step");
      return QFX_OK;
    };
    if (full) {
      // input of step i: site 0's tensor for i = 1, the stored output of step i - 1 after
      for (int i = n - 1; i >= 0; --i) {
        const char* in = i == 0 ? nullptr : i == 1 ? site_ptr(p->steps[0].site) : ckpt(i - 1);
        qfx_status r = reverse_step(i, in);
        if (r != QFX_OK) return r;
      }
    } else {
      // line by line, recomputing each line's inputs from its checkpoint
      for (int w = W - 1; w >= 0; --w) {
        const int i0 = w * L;
        // input of step i0 + j is lb(j) (j >= 1) or ckpt(w)
        auto line_in = [&](int j) -> const char* {
          if (j == 0) return w == 0 ? nullptr : ckpt(w);
          if (w == 0 && j == 1) return site_ptr(p->steps[0].site);
          return lb(j);
        };
        for (int j = 1; j < L && i0 + j < n; ++j) {
          if (w == 0 && j == 1) continue;           // L_1 is site 0 itself
          err = step_fwd(i0 + j - 1, line_in(j - 1), lb(j));
          if (err) return cuda_fail(err, "qfx_amplitudes_backward: recompute step");
        }
        for (int j = std::min(L, n - i0) - 1; j >= 0; --j) {
          qfx_status r = reverse_step(i0 + j, line_in(j));
          if (r != QFX_OK) return r;
        }
      }
    }
    // back through every site's time fold
    dim3 fg((unsigned)((max_site + kT - 1) / kT), n);
    fold_backward_kernel<<<fg, kT, 0, st>>>(t.sites, t.events, t.matsf, t.cuts, (int)p->cut_dev.size(),
                                            x1 + b * p->x1_words, sid, sgrad, (double*)(ws + Lw.bpart),
                                            t.partoff);
    const int nev = (int)p->events.size();
    event_reduce_kernel<<<(nev * 32 + kT - 1) / kT, kT, 0, st>>>(t.sites, n, t.events,
                                                                (const double*)(ws + Lw.bpart),
                                                                t.partoff, exps,
                                                                m_ptr, nev, (double*)(ws + Lw.evgrad));
    gate_accum_kernel<<<(p->n_gates * 2 * per_gate + kT - 1) / kT, kT, 0, st>>>(
        t.gate_ev, t.events, p->n_gates, per_gate, (const double*)(ws + Lw.evgrad), grad_gates);
    count_launch(3);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "qfx_amplitudes_backward: fold adjoint");
  }
  return QFX_OK;
}

}  // namespace

extern "C" qfx_status qfx_amplitudes_backward(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                              int64_t slice_begin, int64_t slice_end,
                                              const double* grad_out, double* grad_gates,
                                              void* workspace, size_t ws_bytes, void* stream) {
  return backward(p, x1, n_batch, slice_begin, slice_end, grad_out, grad_gates, 4, workspace,
                  ws_bytes, stream);
}

extern "C" qfx_status qfx_amplitudes_backward_full(const qfx_plan* p, const uint64_t* x1,
                                                   int64_t n_batch, int64_t slice_begin,
                                                   int64_t slice_end, const double* grad_out,
                                                   double* grad_gates, void* workspace,
                                                   size_t ws_bytes, void* stream) {
  return backward(p, x1, n_batch, slice_begin, slice_end, grad_out, grad_gates, 16, workspace,
                  ws_bytes, stream);
}
