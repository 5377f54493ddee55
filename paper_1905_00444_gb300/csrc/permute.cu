// Tensor transpose for complex64 tensors of rank <= 10 (the "T" steps of TTGT,
// Sec. III.E).  Axes that stay adjacent are fused first.  If the innermost output axis
// is also innermost in the input, rows are copied with 16-byte vectors; otherwise a
// 32 x 32 tile of (output-innermost axis, input-innermost axis) goes through shared
// memory so that both the reads and the writes are coalesced.
#include <cuda_runtime.h>

#include <cstring>

#include "qfx_internal.h"

namespace qfx {
namespace {

constexpr int kMaxRank = 10;

struct PermArgs {
  int rank;                 // fused rank
  int64_t dim[kMaxRank];    // output axis sizes (fused)
  int64_t istr[kMaxRank];   // input stride of each output axis
  int64_t ostr[kMaxRank];   // output stride of each output axis
  int la, lb;               // tiled: la = innermost output axis, lb = axis with input stride 1
  int64_t tiles_a, tiles_b;
};

// ---- case 1: innermost axis shared -> contiguous rows ------------------------
__global__ void __launch_bounds__(256) permute_rows_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a, int64_t rows,
                                                           int64_t chunks) {
  const int64_t row = blockIdx.x / chunks;
  const int64_t chunk = blockIdx.x % chunks;
  if (row >= rows) return;
  const int64_t D = a.dim[a.rank - 1];
  int64_t r = row, ib = 0, ob = 0;
  for (int ax = a.rank - 2; ax >= 0; --ax) {
    const int64_t c = r % a.dim[ax];
    r /= a.dim[ax];
    ib += c * a.istr[ax];
    ob += c * a.ostr[ax];
  }
  const int64_t base = chunk * 512;
  const bool vec = (D % 2 == 0) && (ib % 2 == 0) && (ob % 2 == 0);
  if (vec) {
    const int64_t e = base + 2 * threadIdx.x;
    if (e < D)
      *reinterpret_cast<float4*>(out + ob + e) = *reinterpret_cast<const float4*>(in + ib + e);
  } else {
    for (int64_t e = base + threadIdx.x; e < base + 512 && e < D; e += 256) out[ob + e] = in[ib + e];
  }
}

// ---- case 2: tiled transpose -------------------------------------------------
__global__ void __launch_bounds__(256) permute_tile_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a) {
  __shared__ float2 tile[32][33];
  const int64_t per = a.tiles_a * a.tiles_b;
  const int64_t bidx = blockIdx.x / per;
  const int64_t t = blockIdx.x % per;
  const int64_t ta = t % a.tiles_a, tb = t / a.tiles_a;
  int64_t r = bidx, ib = 0, ob = 0;
  for (int ax = a.rank - 1; ax >= 0; --ax) {
    if (ax == a.la || ax == a.lb) continue;
    const int64_t c = r % a.dim[ax];
    r /= a.dim[ax];
    ib += c * a.istr[ax];
    ob += c * a.ostr[ax];
  }
  const int64_t A0 = ta * 32, B0 = tb * 32;
  const int64_t Da = a.dim[a.la], Db = a.dim[a.lb];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  // read: consecutive x walk the input-innermost axis lb
  for (int yy = y; yy < 32; yy += 8) {
    const int64_t ia = A0 + yy, jb = B0 + x;
    if (ia < Da && jb < Db) tile[yy][x] = in[ib + ia * a.istr[a.la] + jb];
  }
  __syncthreads();
  // write: consecutive x walk the output-innermost axis la
  for (int yy = y; yy < 32; yy += 8) {
    const int64_t jb = B0 + yy, ia = A0 + x;
    if (ia < Da && jb < Db) out[ob + ia + jb * a.ostr[a.lb]] = tile[x][yy];
  }
}

}  // namespace

int launch_permute(const void* in, void* out, int rank, const int64_t* shape,
                   const int32_t* perm, void* stream) {
  if (rank < 1 || rank > kMaxRank) return (int)cudaErrorInvalidValue;
  int64_t istride[kMaxRank];
  istride[rank - 1] = 1;
  for (int i = rank - 2; i >= 0; --i) istride[i] = istride[i + 1] * shape[i + 1];
  int64_t total = 1;
  for (int i = 0; i < rank; ++i) total *= shape[i];
  if (total == 0) return 0;
  // fuse output axes a, a+1 when they are adjacent input axes in the same order
  PermArgs a{};
  int fr = 0;
  for (int i = 0; i < rank; ++i) {
    const int ax = perm[i];
    if (shape[ax] == 1) continue;
    if (fr > 0 && a.istr[fr - 1] == istride[ax] * shape[ax]) {
      a.dim[fr - 1] *= shape[ax];
      a.istr[fr - 1] = istride[ax];
    } else {
      a.dim[fr] = shape[ax];
      a.istr[fr] = istride[ax];
      ++fr;
    }
  }
  if (fr == 0) { a.dim[0] = 1; a.istr[0] = 1; fr = 1; }
  a.rank = fr;
  a.ostr[fr - 1] = 1;
  for (int i = fr - 2; i >= 0; --i) a.ostr[i] = a.ostr[i + 1] * a.dim[i + 1];
  cudaStream_t st = (cudaStream_t)stream;
  const float2* src = (const float2*)in;
  float2* dst = (float2*)out;
  if (a.istr[fr - 1] == 1) {
    const int64_t D = a.dim[fr - 1];
    const int64_t rows = total / D;
    const int64_t chunks = (D + 511) / 512;
    if (rows * chunks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
    permute_rows_kernel<<<(unsigned)(rows * chunks), 256, 0, st>>>(src, dst, a, rows, chunks);
  } else {
    a.la = fr - 1;
    a.lb = -1;
    for (int i = 0; i < fr; ++i)
      if (a.istr[i] == 1) a.lb = i;
    if (a.lb < 0) return (int)cudaErrorInvalidValue;
    a.tiles_a = (a.dim[a.la] + 31) / 32;
    a.tiles_b = (a.dim[a.lb] + 31) / 32;
    const int64_t batch = total / (a.dim[a.la] * a.dim[a.lb]);
    const int64_t blocks = batch * a.tiles_a * a.tiles_b;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
    permute_tile_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a);
  }
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace qfx
