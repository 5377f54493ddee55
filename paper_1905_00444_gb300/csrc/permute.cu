// Tensor transpose for complex64 tensors of rank <= 10 (the "T" steps of TTGT,
// Sec. III.E).  Axes that stay adjacent are fused first.  If the innermost output axis
// is also innermost in the input, rows are copied with 16-byte vectors, 4096 output
// elements per block; otherwise a 32 x 32 tile of (output-innermost axis,
// input-innermost axis) goes through shared memory so that both the reads and the
// writes are coalesced, each block walking 8 consecutive batch coordinates.
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
// Each block copies 4096 consecutive output elements (any number of rows): thread pairs
// of elements stay in one row when D is even, so they move as 16-byte vectors.
constexpr int kRowChunk = 4096;
__global__ void __launch_bounds__(256) permute_rows_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a, int64_t total) {
  const int64_t D = a.dim[a.rank - 1];
  const int64_t base = (int64_t)blockIdx.x * kRowChunk;
  const bool even = (D % 2) == 0;
#pragma unroll 2
  for (int k = 0; k < kRowChunk / 512; ++k) {
    const int64_t o = base + k * 512 + 2 * threadIdx.x;
    if (o >= total) break;
    int64_t row = o / D;
    const int64_t col = o - row * D;
    int64_t ib = 0;
    for (int ax = a.rank - 2; ax >= 0; --ax) {
      const int64_t c = row % a.dim[ax];
      row /= a.dim[ax];
      ib += c * a.istr[ax];
    }
    if (even && (ib % 2) == 0) {
      *reinterpret_cast<float4*>(out + o) = *reinterpret_cast<const float4*>(in + ib + col);
    } else {
      out[o] = in[ib + col];
      if (o + 1 < total) {
        if (col + 1 < D) {
          out[o + 1] = in[ib + col + 1];
        } else {   // next element starts the next row
          int64_t r2 = (o + 1) / D, ib2 = 0;
          for (int ax = a.rank - 2; ax >= 0; --ax) {
            const int64_t c = r2 % a.dim[ax];
            r2 /= a.dim[ax];
            ib2 += c * a.istr[ax];
          }
          out[o + 1] = in[ib2];
        }
      }
    }
  }
}

// ---- case 2: tiled transpose -------------------------------------------------
// A block handles kTileBatch consecutive batch coordinates of one (a, b) tile position,
// stepping the batch odometer instead of decomposing every tile's index.
constexpr int kTileBatch = 8;
__global__ void __launch_bounds__(256) permute_tile_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a, int64_t batch) {
  __shared__ float2 tile[32][33];
  const int64_t per = a.tiles_a * a.tiles_b;
  const int64_t t = blockIdx.x % per;
  const int64_t b0 = (int64_t)(blockIdx.x / per) * kTileBatch;
  const int64_t ta = t % a.tiles_a, tb = t / a.tiles_a;
  // batch coordinates of b0
  int64_t coord[kMaxRank];
  int64_t r = b0, ib = 0, ob = 0;
  for (int ax = a.rank - 1; ax >= 0; --ax) {
    coord[ax] = 0;
    if (ax == a.la || ax == a.lb) continue;
    coord[ax] = r % a.dim[ax];
    r /= a.dim[ax];
    ib += coord[ax] * a.istr[ax];
    ob += coord[ax] * a.ostr[ax];
  }
  const int64_t A0 = ta * 32, B0 = tb * 32;
  const int64_t Da = a.dim[a.la], Db = a.dim[a.lb];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  for (int64_t bi = b0; bi < b0 + kTileBatch && bi < batch; ++bi) {
    for (int yy = y; yy < 32; yy += 8) {
      const int64_t ia = A0 + yy, jb = B0 + x;
      if (ia < Da && jb < Db) tile[yy][x] = in[ib + ia * a.istr[a.la] + jb];
    }
    __syncthreads();
    for (int yy = y; yy < 32; yy += 8) {
      const int64_t jb = B0 + yy, ia = A0 + x;
      if (ia < Da && jb < Db) out[ob + ia + jb * a.ostr[a.lb]] = tile[x][yy];
    }
    __syncthreads();
    // odometer: next batch coordinate (innermost batch axis first)
    for (int ax = a.rank - 1; ax >= 0; --ax) {
      if (ax == a.la || ax == a.lb) continue;
      ib += a.istr[ax];
      ob += a.ostr[ax];
      if (++coord[ax] < a.dim[ax]) break;
      ib -= coord[ax] * a.istr[ax];
      ob -= coord[ax] * a.ostr[ax];
      coord[ax] = 0;
    }
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
    const int64_t blocks = (total + kRowChunk - 1) / kRowChunk;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
    permute_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a, total);
  } else {
    a.la = fr - 1;
    a.lb = -1;
    for (int i = 0; i < fr; ++i)
      if (a.istr[i] == 1) a.lb = i;
    if (a.lb < 0) return (int)cudaErrorInvalidValue;
    a.tiles_a = (a.dim[a.la] + 31) / 32;
    a.tiles_b = (a.dim[a.lb] + 31) / 32;
    const int64_t batch = total / (a.dim[a.la] * a.dim[a.lb]);
    const int64_t blocks = ((batch + kTileBatch - 1) / kTileBatch) * a.tiles_a * a.tiles_b;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
    permute_tile_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a, batch);
  }
  count_launch();
  return (int)cudaGetLastError();
}

}  // namespace qfx
