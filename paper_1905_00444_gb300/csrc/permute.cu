// Tensor transpose for complex64 tensors of rank <= 10 (the "T" steps of TTGT,
// Sec. III.E).  Axes that stay adjacent are fused first.
// - Innermost output axis also innermost in the input: rows are copied with 16-byte
//   vectors, 4096 output elements per block.
// - Otherwise, when both innermost axes have at least 16 elements and the strides allow
//   a tensor map: tiles of 16 (input-innermost axis lb) x TA (output-innermost axis la)
//   x BZ (consecutive values of one more axis) elements arrive by tensor-map copies with
//   128-byte swizzle into a ring of shared buffers; each warp instruction then reads 16
//   consecutive la by 2 consecutive lb (conflict-free under the swizzle) and writes two
//   128-byte output segments.  The input is viewed as a 5-D tensor: lb, la, and the
//   other axes merged into at most three runs that are contiguous in the input.
// - Otherwise a 32 x 32 tile goes through shared memory with plain loads, each block
//   walking 8 consecutive batch coordinates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ptx_async.cuh"
#include "qfx_internal.h"

namespace qfx {

__device__ unsigned int g_perm_status = 0;

namespace {

using namespace ptx;

constexpr int kMaxRank = 10;

struct PermArgs {
  int rank;                 // fused rank
  int64_t dim[kMaxRank];    // output axis sizes (fused)
  int64_t istr[kMaxRank];   // input stride of each output axis
  int64_t ostr[kMaxRank];   // output stride of each output axis
  int la, lb;               // tiled: la = innermost output axis, lb = axis with input stride 1
  int64_t tiles_a, tiles_b;
  int na;                   // tiled: the tile's a side spans the last na output axes (not lb)
  int64_t da;               // their extent (contiguous in the output)
};

// ---- case 1: innermost axis shared -> contiguous rows ------------------------
// Each block copies 4096 consecutive output elements (any number of rows): thread pairs
// of elements stay in one row when D is even, so they move as 16-byte vectors.  The
// input offset of every row the block touches is computed once into shared memory: each
// thread takes a run of consecutive rows, decomposes the first one (mixed-radix
// divisions) and steps an odometer through the rest.
constexpr int kRowChunk = 4096;
constexpr int kMaxChunkRows = kRowChunk / 2 + 2;   // D >= 2 for this kernel
__global__ void __launch_bounds__(256) permute_rows_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a, int64_t total) {
  __shared__ int64_t rowoff[kMaxChunkRows];
  const int64_t D = a.dim[a.rank - 1];
  const int64_t base = (int64_t)blockIdx.x * kRowChunk;
  const int64_t r0 = base / D;
  const int64_t end = min(total, base + kRowChunk);
  const int nrows = (int)((end - 1) / D - r0 + 1);
  const int per = (nrows + (int)blockDim.x - 1) / (int)blockDim.x;
  const int i0 = (int)threadIdx.x * per, i1 = min(nrows, i0 + per);
  if (i0 < i1) {
    int64_t coord[kMaxRank];
    int64_t row = r0 + i0, ib = 0;
    for (int ax = a.rank - 2; ax >= 0; --ax) {
      coord[ax] = row % a.dim[ax];
      row /= a.dim[ax];
      ib += coord[ax] * a.istr[ax];
    }
    for (int i = i0; i < i1; ++i) {
      rowoff[i] = ib;
      for (int ax = a.rank - 2; ax >= 0; --ax) {   // the next row
        ib += a.istr[ax];
        if (++coord[ax] < a.dim[ax]) break;
        ib -= coord[ax] * a.istr[ax];
        coord[ax] = 0;
      }
    }
  }
  __syncthreads();
  const int Di = (int)D, first = (int)(base - r0 * D);   // column of the block's first element
  const bool even = (D % 2) == 0;
#pragma unroll 2
  for (int k = 0; k < kRowChunk / 512; ++k) {
    const int lo = k * 512 + 2 * threadIdx.x;   // element offset inside the chunk
    const int64_t o = base + lo;
    if (o >= total) break;
    const int rl = (first + lo) / Di, col = first + lo - rl * Di;
    const int64_t ib = rowoff[rl];
    if (even && (ib % 2) == 0) {
      *reinterpret_cast<float4*>(out + o) = *reinterpret_cast<const float4*>(in + ib + col);
    } else {
      out[o] = in[ib + col];
      if (o + 1 < total) out[o + 1] = col + 1 < Di ? in[ib + col + 1] : in[rowoff[rl + 1]];
    }
  }
}

// Rows of one element (or longer than 2^30): the mixed-radix divisions stay per element.
__global__ void __launch_bounds__(256) permute_short_rows_kernel(const float2* __restrict__ in,
                                                                 float2* __restrict__ out,
                                                                 const PermArgs a, int64_t total) {
  const int64_t D = a.dim[a.rank - 1];
  const int64_t o = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (o >= total) return;
  int64_t row = o / D, ib = 0;
  const int64_t col = o - row * D;
  for (int ax = a.rank - 2; ax >= 0; --ax) {
    const int64_t c = row % a.dim[ax];
    row /= a.dim[ax];
    ib += c * a.istr[ax];
  }
  out[o] = in[ib + col];
}

// ---- case 2: tiled transpose -------------------------------------------------
// A block handles kTileBatch consecutive batch coordinates of one (a, b) tile position,
// stepping the batch odometer instead of decomposing every tile's index.
constexpr int kTileBatch = 8;
__global__ void __launch_bounds__(256) permute_tile_kernel(const float2* __restrict__ in,
                                                           float2* __restrict__ out,
                                                           const PermArgs a, int64_t batch) {
  __shared__ float2 tile[32][33];
  __shared__ int64_t offa[32];
  const int64_t per = a.tiles_a * a.tiles_b;
  const int64_t t = blockIdx.x % per;
  const int64_t b0 = (int64_t)(blockIdx.x / per) * kTileBatch;
  const int64_t ta = t % a.tiles_a, tb = t / a.tiles_a;
  // batch coordinates of b0
  int64_t coord[kMaxRank];
  int64_t r = b0, ib = 0, ob = 0;
  const int afirst = a.rank - a.na;   // the a side: output axes afirst .. rank-1
  for (int ax = a.rank - 1; ax >= 0; --ax) {
    coord[ax] = 0;
    if (ax >= afirst || ax == a.lb) continue;
    coord[ax] = r % a.dim[ax];
    r /= a.dim[ax];
    ib += coord[ax] * a.istr[ax];
    ob += coord[ax] * a.ostr[ax];
  }
  const int64_t A0 = ta * 32, B0 = tb * 32;
  const int64_t Da = a.da, Db = a.dim[a.lb];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  if (threadIdx.x < 32) {   // input offsets of the tile's 32 positions along a
    int64_t ia = A0 + threadIdx.x, off = 0;
    if (ia < Da)
      for (int ax = a.rank - 1; ax >= afirst; --ax) {
        off += (ia % a.dim[ax]) * a.istr[ax];
        ia /= a.dim[ax];
      }
    offa[threadIdx.x] = off;
  }
  __syncthreads();
  for (int64_t bi = b0; bi < b0 + kTileBatch && bi < batch; ++bi) {
    for (int yy = y; yy < 32; yy += 8) {
      const int64_t ia = A0 + yy, jb = B0 + x;
      if (ia < Da && jb < Db) tile[yy][x] = in[ib + offa[yy] + jb];
    }
    __syncthreads();
    for (int yy = y; yy < 32; yy += 8) {
      const int64_t jb = B0 + yy, ia = A0 + x;
      if (ia < Da && jb < Db) out[ob + ia + jb * a.ostr[a.lb]] = tile[x][yy];
    }
    __syncthreads();
    // odometer: next batch coordinate (innermost batch axis first)
    for (int ax = a.rank - 1; ax >= 0; --ax) {
      if (ax >= afirst || ax == a.lb) continue;
      ib += a.istr[ax];
      ob += a.ostr[ax];
      if (++coord[ax] < a.dim[ax]) break;
      ib -= coord[ax] * a.istr[ax];
      ob -= coord[ax] * a.ostr[ax];
      coord[ax] = 0;
    }
  }
}


// ---- case 3: tensor-map staged transpose -------------------------------------------
struct PermTma {
  int64_t Da, Db;           // extents of la (output stride 1) and lb (input stride 1)
  int64_t tiles_a, tiles_b, nbatch, total;
  int64_t ostr_b;           // output stride of lb
  int nseg;                 // runs of the other axes, contiguous in the input (<= 3)
  int64_t segE[3];          // run extents (coordinates 2..4 of the tensor map)
  int seg_n[3];             // axes per run, innermost first
  int64_t ax_dim[kMaxRank], ax_ostr[kMaxRank];   // the runs' axes, run by run
  int BZ;                   // box extent along run 0 (divides its innermost axis)
  int64_t tiles_z;          // segE[0] / BZ (1 if there is no run)
  int64_t ostr_z;           // output stride of run 0's innermost axis
  unsigned long long wait_ns;   // limit of every bounded wait
  int withhold;             // test hook: issue no copies (every consumer's wait runs out)
};
constexpr unsigned long long kPermWaitNs = 1000000000ull;   // 1 s per wait
// test hook (qfx_debug_permute_withhold): the next tensor-map permute of this thread
// issues no copies and waits at most this long
thread_local unsigned long long g_perm_withhold_ns = 0;

struct TileMeta {
  int64_t obase;
  int na, nb;
};

// Thread 0: tensor-map coordinates and output placement of tile t; issues its copy.
template <int TA>
__device__ __forceinline__ void perm_issue(const PermTma& a, const CUtensorMap* map, int64_t t, uint32_t dst,
                                           uint32_t bar, TileMeta* meta) {
  constexpr int TB = 16;
  const int64_t ta = t % a.tiles_a, r = t / a.tiles_a;
  const int64_t tb = r % a.tiles_b;
  int64_t bi = r / a.tiles_b;
  int z[3] = {0, 0, 0};
  int64_t obase = ta * TA + tb * TB * a.ostr_b;
  for (int g = a.nseg - 1; g >= 1; --g) {   // run 0 most significant
    const int64_t zg = bi % a.segE[g];
    bi /= a.segE[g];
    z[g] = (int)zg;
  }
  if (a.nseg > 0) z[0] = (int)(bi * a.BZ);  // run 0 advances a box of BZ at a time
  int ax = 0;
  for (int g = 0; g < a.nseg; ++g) {
    int64_t zg = z[g];
    for (int i = 0; i < a.seg_n[g]; ++i, ++ax) {
      const int64_t c = zg % a.ax_dim[ax];
      zg /= a.ax_dim[ax];
      obase += c * a.ax_ostr[ax];
    }
  }
  meta->obase = obase;
  const int64_t ra = a.Da - ta * TA, rb = a.Db - tb * TB;
  meta->na = (int)(ra < TA ? ra : TA);
  meta->nb = (int)(rb < TB ? rb : TB);
  mbar_arrive_tx(bar, (uint32_t)(TB * TA * a.BZ * 8));
  tma_load_5d(dst, map, (int)(tb * TB), (int)(ta * TA), z[0], z[1], z[2], bar);
}

// Warps 0-3 consume tiles; lane 0 of warp 4 issues the copies NB tiles ahead, reusing a
// buffer once its 128 consumers have released it.  Every wait is bounded; a timeout sets
// the status word and makes the other roles give up too.
template <int TA, int NB>
__global__ void __launch_bounds__(160) permute_tma_kernel(const PermTma a, float2* __restrict__ out,
                                                          const __grid_constant__ CUtensorMap map) {
  constexpr int TB = 16;
  const int TILE = TB * TA * 8 * a.BZ, UNITS = 8 * (TA / 16) * a.BZ;
  extern __shared__ char smem_raw[];
  // 128-byte swizzled boxes must start on 1024-byte boundaries
  char* buf = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[NB], empty[NB];
  __shared__ TileMeta meta[NB];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int b = 0; b < NB; ++b) {
      mbar_init(smem_u32(&full[b]), 1);
      mbar_init(smem_u32(&empty[b]), 128);
    }
    abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();
  volatile int* abort = &abort_flag;
  auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long deadline = globaltimer() + a.wait_ns;
    while (!mbar_try(bar, parity)) {
      if (*abort) return false;
      if (globaltimer() > deadline) {
        *abort = 1;
        atomicOr(&g_perm_status, 1u);
        return false;
      }
    }
    return true;
  };
  const int64_t stride = gridDim.x;
  if (warp == 4) {
    if (lane == 0) {
      int64_t k = 0, issued = 0;
      for (int64_t t = blockIdx.x; t < a.total; t += stride, ++k) {
        const int b = (int)(k % NB);
        if (a.withhold) break;
        if (k >= NB && !wait(smem_u32(&empty[b]), (uint32_t)((k / NB - 1) & 1))) break;
        perm_issue<TA>(a, &map, t, smem_u32(buf + b * TILE), smem_u32(&full[b]), &meta[b]);
        issued = k + 1;
      }
      // copies still in flight must land before the block exits
      for (int64_t i = (issued > NB ? issued - NB : 0); i < issued; ++i) {
        const int b = (int)(i % NB);
        const unsigned long long deadline = globaltimer() + a.wait_ns;
        while (!mbar_try(smem_u32(&full[b]), (uint32_t)((i / NB) & 1)) && globaltimer() < deadline) {
        }
      }
    }
    return;
  }
  const int ia_lo = lane & 15, h = lane >> 4;
  int64_t k = 0;
  for (int64_t t = blockIdx.x; t < a.total; t += stride, ++k) {
    const int b = (int)(k % NB);
    if (!wait(smem_u32(&full[b]), (uint32_t)((k / NB) & 1))) break;
    const TileMeta m = meta[b];
    const char* tile = buf + b * TILE;
    for (int u = warp; u < UNITS; u += 4) {
      const int c = u & 7, iz = (u >> 3) / (TA / 16), ia = ((u >> 3) % (TA / 16)) * 16 + ia_lo, ib = 2 * c + h;
      // row (iz, ia) of the box is 128 bytes of lb; its 16-byte chunk c sits at
      // c ^ (row mod 8), and row mod 8 = ia mod 8 since TA is a multiple of 8
      const float2 v = *reinterpret_cast<const float2*>(tile + (iz * TA + ia) * 128 + ((c ^ (ia & 7)) << 4) + h * 8);
      if (ia < m.na && ib < m.nb) out[m.obase + iz * a.ostr_z + ia + (int64_t)ib * a.ostr_b] = v;
    }
    // the next copy into this buffer goes through the async proxy: order the reads first
    fence_async_smem();
    mbar_arrive(smem_u32(&empty[b]));
  }
}

// Host: the 5-D view and tensor map of the input, or false when this path does not apply.
bool perm_tma_plan(const PermArgs& f, const void* in, PermTma* t, CUtensorMap* map, int* ta_out) {
  auto enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)in & 15)) return false;
  const int fr = f.rank, la = f.la, lb = f.lb;
  const int64_t Da = f.dim[la], Db = f.dim[lb];
  if (Da < 16 || Db < 16 || Da > 0x7fffffff || Db > 0x7fffffff) return false;
  // the other axes in input order (outermost first), cut into runs contiguous in the input
  int order[kMaxRank], n = 0;
  for (int i = 0; i < fr; ++i)
    if (i != la && i != lb) order[n++] = i;
  for (int i = 1; i < n; ++i)   // sort by input stride, descending
    for (int j = i; j > 0 && f.istr[order[j]] > f.istr[order[j - 1]]; --j) std::swap(order[j], order[j - 1]);
  PermTma a{};
  a.Da = Da;
  a.Db = Db;
  a.ostr_b = f.ostr[lb];
  int64_t segS[3] = {1, 1, 1};
  int ax = 0;
  for (int i = 0; i < n;) {
    if (a.nseg == 3) return false;
    int j = i;   // run [i, j]: each next axis sits right inside the previous one in memory
    while (j + 1 < n && f.istr[order[j]] == f.istr[order[j + 1]] * f.dim[order[j + 1]]) ++j;
    int64_t E = 1;
    for (int q = j; q >= i; --q) {   // innermost first
      a.ax_dim[ax] = f.dim[order[q]];
      a.ax_ostr[ax] = f.ostr[order[q]];
      ++ax;
      E *= f.dim[order[q]];
    }
    if (E > 0x7fffffff) return false;
    a.segE[a.nseg] = E;
    a.seg_n[a.nseg] = j - i + 1;
    segS[a.nseg] = f.istr[order[j]];
    ++a.nseg;
    i = j + 1;
  }
  // strides of map dimensions 1..4 in bytes must be multiples of 16
  if ((f.istr[la] & 1) || (a.nseg > 0 && (segS[0] & 1)) || (a.nseg > 1 && (segS[1] & 1)) ||
      (a.nseg > 2 && (segS[2] & 1)))
    return false;
  const int TA = Da >= 64 ? 64 : Da >= 32 ? 32 : 16;
  a.tiles_a = (Da + TA - 1) / TA;
  a.tiles_b = (Db + 15) / 16;
  // boxes of 8 KB or more: BZ values of run 0's innermost axis (a divisor of its extent)
  a.BZ = 1;
  a.ostr_z = 0;
  if (a.nseg > 0) {
    const int want = 64 / TA;   // 1, 2 or 4 ... up to 8 for TA = 16
    const int64_t d0 = a.ax_dim[0];   // run 0's innermost axis
    int bz = 1;
    while (bz * 2 <= (TA == 16 ? 8 : want) && d0 % (bz * 2) == 0) bz *= 2;
    a.BZ = bz;
    a.ostr_z = a.ax_ostr[0];
  }
  a.nbatch = 1;
  for (int g = 1; g < a.nseg; ++g) a.nbatch *= a.segE[g];
  if (a.nseg > 0) a.nbatch *= a.segE[0] / a.BZ;
  a.total = a.tiles_a * a.tiles_b * a.nbatch;
  a.wait_ns = kPermWaitNs;
  a.withhold = 0;
  int64_t total_el = 1;
  for (int i = 0; i < fr; ++i) total_el *= f.dim[i];
  const cuuint64_t pad_stride = (cuuint64_t)((total_el * 8 + 15) / 16 * 16);
  cuuint64_t dims[5] = {(cuuint64_t)Db, (cuuint64_t)Da, 1, 1, 1};
  cuuint64_t strides[4] = {(cuuint64_t)f.istr[la] * 8, pad_stride, pad_stride, pad_stride};
  for (int g = 0; g < a.nseg; ++g) {
    dims[2 + g] = (cuuint64_t)a.segE[g];
    strides[1 + g] = (cuuint64_t)segS[g] * 8;
  }
  const cuuint32_t box[5] = {16, (cuuint32_t)TA, (cuuint32_t)a.BZ, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(in), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  *t = a;
  *ta_out = TA;
  return true;
}

template <int TA, int NB>
int launch_perm_tma(const PermTma& a, const CUtensorMap& map, float2* out, cudaStream_t st) {
  const size_t smem = (size_t)NB * 16 * TA * 8 * a.BZ + 1024;   // NB x 8 or 16 KB
  static int attr_dev[64] = {0};
  int dev0 = 0;
  cudaGetDevice(&dev0);
  if (dev0 < 64 && !attr_dev[dev0]) {
    cudaError_t e = cudaFuncSetAttribute(permute_tma_kernel<TA, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         NB * 16384 + 1024);   // boxes are at most 16 KB
    if (e != cudaSuccess) return (int)e;
    attr_dev[dev0] = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // as many blocks per SM as 220 KB of shared memory holds, at most 8
  int per_sm = (int)((220u << 10) / (smem + 512));
  per_sm = per_sm < 1 ? 1 : per_sm > 8 ? 8 : per_sm;
  const int64_t want = (int64_t)(sms > 0 ? sms : 1) * per_sm;
  const unsigned grid = (unsigned)(a.total < want ? a.total : want);
  permute_tma_kernel<TA, NB><<<grid, 160, smem, st>>>(a, out, map);
  return (int)cudaGetLastError();
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
    if (a.dim[fr - 1] >= 2 && a.dim[fr - 1] < (int64_t(1) << 30)) {
      const int64_t blocks = (total + kRowChunk - 1) / kRowChunk;
      if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
      permute_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a, total);
    } else {
      const int64_t blocks = (total + 255) / 256;
      if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
      permute_short_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a, total);
    }
  } else {
    a.la = fr - 1;
    a.lb = -1;
    for (int i = 0; i < fr; ++i)
      if (a.istr[i] == 1) a.lb = i;
    if (a.lb < 0) return (int)cudaErrorInvalidValue;
    PermTma tp;
    alignas(64) CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    int TA = 0;
    if (perm_tma_plan(a, in, &tp, &map, &TA)) {
      if (g_perm_withhold_ns) {   // test hook, one call only
        tp.withhold = 1;
        tp.wait_ns = g_perm_withhold_ns;
        g_perm_withhold_ns = 0;
      }
      const int err = TA == 64 ? launch_perm_tma<64, 4>(tp, map, dst, st)
                    : TA == 32 ? launch_perm_tma<32, 4>(tp, map, dst, st)
                               : launch_perm_tma<16, 4>(tp, map, dst, st);
      count_launch();
      return err;
    }
    // the tile's a side: the innermost output axis, widened by the next ones outwards
    // (stopping at lb) until it spans 32 elements; they are contiguous in the output
    a.na = 1;
    a.da = a.dim[fr - 1];
    while (a.da < 32 && fr - 1 - a.na >= 0 && fr - 1 - a.na != a.lb) {
      a.da *= a.dim[fr - 1 - a.na];
      ++a.na;
    }
    a.tiles_a = (a.da + 31) / 32;
    a.tiles_b = (a.dim[a.lb] + 31) / 32;
    const int64_t batch = total / (a.da * a.dim[a.lb]);
    const int64_t blocks = ((batch + kTileBatch - 1) / kTileBatch) * a.tiles_a * a.tiles_b;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidConfiguration;
    permute_tile_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, a, batch);
  }
  count_launch();
  return (int)cudaGetLastError();
}

int perm_take_status() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_perm_status, sizeof(v)) != cudaSuccess) return -1;
  if (v) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_perm_status, &z, sizeof(z));
  }
  return v ? 1 : 0;
}

}  // namespace qfx

extern "C" qfx_status qfx_debug_permute_withhold(int64_t wait_ns) {
  if (wait_ns < 1000 || wait_ns > 1000000000)
    return qfx::fail(QFX_EINVAL, "qfx_debug_permute_withhold: wait_ns must be in [1e3, 1e9]");
  qfx::g_perm_withhold_ns = (unsigned long long)wait_ns;
  return QFX_OK;
}
