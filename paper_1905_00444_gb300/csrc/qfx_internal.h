// Internal structures of libqfx shared by the host planner and the CUDA kernels.
#pragma once

#include <array>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "qfx.h"

namespace qfx {

constexpr int kMaxSites = 144;   // 12 x 12 grids; bitstrings of more than 64 qubits span several words
constexpr int kMaxOpen = 24;
constexpr int kMaxCuts = 64;

// ---------------------------------------------------------------------------
// circuit
// ---------------------------------------------------------------------------
struct Gate {
  int layer, q0, q1, kind;
  double m[32];
  int index;   // position in the caller's gate list
};

}  // namespace qfx

struct qfx_circuit {
  int rows = 0, cols = 0;
  std::vector<qfx::Gate> gates;   // sorted by layer (stable)
};

namespace qfx {

// ---------------------------------------------------------------------------
// time fold program (Sec. III: contraction in the time direction first)
// ---------------------------------------------------------------------------
enum EventKind : int32_t {
  EV_GATE = 0,   // v <- G v, G = 2x2 matrix `mat`
  EV_PROJ = 1,   // this site is q0 of a diagonal 2q gate: v <- |k><k| v, k = leg bit
  EV_DIAG = 2,   // this site is q1: v <- diag(D[k][0], D[k][1]) v, k = leg bit
  EV_ELEM = 3,   // q0 of a general 2q gate: v <- |k >> 1><k & 1| v, k = the 2-bit leg
  EV_BLOCK = 4   // q1 of a general 2q gate: v <- B_k v, B_k = matrix `mat + k` (4 in a row)
};

struct FoldEvent {
  int32_t kind;
  int32_t slot;   // bond slot 0..3 (up, left, right, down) holding the leg
  int32_t bit;    // lowest bit of the bond value that holds this leg
  int32_t mat;    // index into the matrix table (4 complex doubles each)
  int32_t gate;   // the gate's index in the caller's list (gradients are reported there)
};

// Site tensor layout: T[up][left][x][right][down] (row-major), so that k = (up, left)
// and n = (x, right, down) in the step formula.
struct FoldSite {
  int32_t qubit;
  int32_t ev_begin, ev_end;
  int32_t edge[4];      // edge id per slot (up, left, right, down), -1 if absent
  int32_t dim[5];       // local dims: up, left, x, right, down (after slicing)
  int32_t x_open;       // 1 if the output leg stays open
  int32_t pad;
  int64_t size;         // product of dims
  int64_t offset;       // element offset of this site in an item's site region
};

struct CutDev {
  int32_t edge;
  int32_t size;         // slice width in bond values
  int64_t radix;        // number of pieces
  int64_t suffix;       // product of the radices of later cuts
};

// ---------------------------------------------------------------------------
// contraction steps
// ---------------------------------------------------------------------------
struct Step {
  int32_t site;
  int32_t variant;
  int64_t P, K, N, NL, Sd;
  double flops, bytes;
  int32_t parts;   // tree nodes: split-K partial products (TreeNode::parts)
};

// One node of a contraction-tree plan (plan family 1): C = A * B over their shared legs as
// the step kernel's C[nh][p][nl][s] = sum_k S[k][nh*NL+nl] B[p][k][s] (NL = N), with
// optional permutes of A (to [shared][free]) and of B (to [shared][free]) first.  Offsets
// are bytes within one work item's block; a permute's fused form has at most 10 axes.
constexpr int kTreeMaxRank = 10;
struct TreeNode {
  int32_t a, b, out;                 // tensor ids (sites 0..n-1, then results in node order)
  int32_t permA, permB;              // 1: permute the operand first
  int32_t rankA, rankB;              // fused permute ranks
  int64_t shapeA[kTreeMaxRank], shapeB[kTreeMaxRank];   // fused input shapes
  int32_t ordA[kTreeMaxRank], ordB[kTreeMaxRank];       // out axis a = input axis ord[a]
  int64_t P, K, N, NL, Sd;
  double flops, bytes;
  uint64_t offA, offB, offA2, offB2, offC;
  int32_t variant;
  int64_t chunk;                     // K > kTreeChunk: K is summed in chunks of this many
  int32_t parts;                     // > 0: the chunks' products side by side, then summed
};
// Contractions longer than this run as chunks of this length, each added into the result:
// an FP32 sum's rounding error grows with the square root of its length, and the tree's
// pairwise contractions of large tensors reach K = 2^20.
constexpr int64_t kTreeChunk = 1024;
// A chunked contraction whose result has at most kTreeSplitOut elements fills too few CTAs
// per chunk: its chunks instead run as one launch (one CTA row per chunk) into partial
// products of at most kTreeSplitBytes per item, summed by launch_reduce_parts.
constexpr int64_t kTreeSplitOut = int64_t(1) << 18;
constexpr uint64_t kTreeSplitBytes = uint64_t(64) << 20;

// Workspace layout:
//   header: per concurrent item: maxabs[n_sites] (u32) + exps[n_sites] (i32), padded
//   items : per concurrent item: buf0 (max_elements) | buf1 (max_elements) | sites
struct Layout {
  uint64_t header_per_item;   // bytes
  uint64_t item_bytes;        // bytes, multiple of 256
  uint64_t buf0, buf1, sites; // byte offsets inside one item block
  uint64_t simage;            // pre-split site image for tensor-core steps (0 bytes if none)
};

// A plan's tables as the kernels see them: regions of one image that every compute call
// copies from the plan's host image into the caller's workspace (nothing is allocated).
struct DeviceTables {
  void* base = nullptr;          // start of the image in device memory
  const FoldSite* sites = nullptr;
  const FoldEvent* events = nullptr;
  const double* mats = nullptr;  // [n_mats][8]
  const CutDev* cuts = nullptr;
  const int32_t* open_perm = nullptr;  // output bit i -> bit of the final tensor index
  const int32_t* gate_ev = nullptr;    // per caller gate: its (up to 2) fold events, -1 if none
  const int64_t* partoff = nullptr;    // per site: first fold-adjoint partial of the site
  const float* matsf = nullptr;        // [n_mats][16]: mats' entries as float-float pairs (hi, lo)
};

}  // namespace qfx

struct qfx_plan {
  int rows = 0, cols = 0, n = 0;
  int x1_words = 1;               // uint64 words per bitstring, ceil(n / 64)
  int n_gates = 0;
  int lines = 0, line_len = 0;    // sweep geometry: steps [w*line_len, (w+1)*line_len) form line w
  int precision = 0;
  int tc_flags = 0;
  uint64_t adjoint_store_bytes = 4ull << 30;  // backward keeps all step outputs up to this
  bool transposed = false;        // lines are grid rows instead of columns
  std::vector<int> order;         // qubits in sweep order
  std::vector<int> open_sites;    // user order (output bit i)
  std::vector<int32_t> open_perm; // output bit i -> final tensor bit
  std::vector<int32_t> gate_ev;   // 2 per caller gate
  std::vector<std::pair<int, int>> edges;  // (q_lo, q_hi)
  std::vector<int> edge_legs;     // legs per edge
  std::vector<qfx_cut> cuts;      // in slice-id digit order (first = most significant)
  std::vector<qfx::CutDev> cut_dev;
  int64_t n_slices = 1;
  std::vector<qfx::FoldSite> sites;     // indexed by qubit
  std::vector<qfx::FoldEvent> events;
  std::vector<double> mats;
  std::vector<qfx::Step> steps;   // steps[0] is the free first site
  int64_t max_elements = 1;
  int64_t site_total = 0;
  double flops_per_item = 0, bytes_per_item = 0;
  int largest_step = 0;
  qfx::Layout layout{};
  int family = 0;                 // 0 = line sweep, 1 = contraction tree (nodes below)
  std::vector<qfx::TreeNode> tree;
  uint64_t tree_final_off = 0;    // byte offset of the tree's result in an item block
  // host image of the tables (page-aligned, built once at creation), copied into the
  // caller's workspace by every compute call; page-locked on first use so that the copy
  // is asynchronous and can be recorded into a CUDA graph
  char* timg = nullptr;
  uint64_t timg_bytes = 0;        // image size, multiple of 256 (the workspace region)
  uint64_t timg_alloc = 0;        // allocation size, multiple of the page size
  size_t toffs[8] = {0};          // region offsets (qfx::kTableRegions)
  mutable std::mutex mu;
  mutable bool timg_pinned = false;
  mutable bool timg_tried = false;
};

namespace qfx {

// error reporting (thread-local message)
qfx_status fail(qfx_status st, const std::string& msg);
qfx_status cuda_fail(int err, const char* what);

// kernels (implemented in .cu files); all return 0 or a cudaError_t value
int launch_fold(const DeviceTables& t, int n_sites, int64_t max_site_size, int n_cuts,
                const uint64_t* x1, int x1_words, int64_t n_batch, int64_t slice_begin,
                int64_t item0, int items, char* hdr, uint64_t hdr_stride, char* itemsp,
                uint64_t item_bytes, uint64_t sites_off, void* stream);
int launch_scale(const DeviceTables& t, int n_sites, int64_t max_site_size, int items,
                 char* hdr, uint64_t hdr_stride, char* itemsp, uint64_t item_bytes,
                 uint64_t sites_off, void* stream);
int launch_accumulate(const DeviceTables& t, int n_sites, int n_open, int64_t n_batch,
                      int64_t item0, int items, const char* hdr, uint64_t hdr_stride,
                      const char* itemsp, uint64_t item_bytes, uint64_t final_off, double* out,
                      void* stream);
int launch_step(const void* S, int64_t s_stride, const void* B, int64_t b_stride, void* C,
                int64_t c_stride, int64_t P, int64_t K, int64_t N, int64_t NL, int64_t Sd,
                int batch, int variant, int precision, void* stream, int beta = 0);
int pick_variant(int64_t N, int64_t Sd);
// Per-step launches: variant 0..9 -> its fill variant (20..28) when the grid of `batch`
// entries would leave SMs idle (same results); any other variant unchanged.
int fill_variant(int variant, int64_t N, int64_t J, int batch);
bool simt_variant_valid(int variant, int64_t Sd);
int num_sms();
// C[b][e] = sum over c < parts of part[b][c][e] (e < out; complex FP32 in and out), per batch
// entry b < batch, in FP64 and a fixed order; strides in float2 units.
int launch_reduce_parts(const void* part, int64_t part_stride, int64_t parts, int64_t out, void* C,
                        int64_t c_stride, int batch, void* stream);
// tensor-core steps (variants 10 = BF16x3, 11 = TF32x3)
constexpr int kVariantTcBf16 = 10, kVariantTcTf32 = 11, kVariantTcBf16x2 = 14;
constexpr int kTcFast = 1;       // QFX_TC_FAST_ACCUMULATION
constexpr int kTcWithhold = 2;   // test hook: S stream withheld
constexpr int kTcNoTma = 4;      // QFX_TC_REGISTER_ROWS
constexpr int kTcBeta = 8;       // add the product into C instead of writing it
bool tc_eligible(int precision, int64_t K, int64_t N, int64_t J, int flags);
uint64_t tc_scratch_bytes(int precision, int64_t K, int64_t N);
int launch_step_tc(const void* S, int64_t s_stride, const void* B, int64_t b_stride, void* C,
                   int64_t c_stride, int64_t P, int64_t K, int64_t N, int64_t NL, int64_t Sd,
                   int batch, int precision, char* scratch, int64_t scratch_stride, void* stream,
                   int flags = 0);

int tc_take_status();     // reads and clears the tensor-core kernels' timeout flag
int tc_probe(int precision, int64_t iters, double* tflops, void* stream);
int tc_prepare_attributes();     // shared-memory opt-ins of every tensor-core kernel
int simt_prepare_attributes();   // and of every FP32 tile kernel
int batch_take_status();  // reads and clears the batch scheduler's timeout flag
uint64_t graph_lane_bytes(const qfx_batch_item* items, int32_t n_items);
int perm_take_status();   // reads and clears the permute kernel's timeout flag
int launch_permute(const void* in, void* out, int rank, const int64_t* shape,
                   const int32_t* perm, void* stream);

void apply_autotune_cache(qfx_plan* p, const char* path);
int tc_variant_of(int precision);   // plan-step variant marking a tensor-core step

// A plan's tables: regions sites, events, mats, cuts, open_perm, gate_ev, partoff, matsf
// of one image.  build_table_image packs the host image at plan creation; stage_tables copies it
// (asynchronously on `stream`) to `dst`, a 256-byte aligned region of table_bytes(p) bytes
// of the caller's workspace, and returns the kernels' view of it.
constexpr int kTableRegions = 8;
void build_table_image(qfx_plan* p);
void free_table_image(qfx_plan* p);
inline uint64_t table_bytes(const qfx_plan* p) { return p->timg_bytes; }
qfx_status pin_tables(const qfx_plan* p);   // page-locks the host image (once; see qfx_plan_upload)
qfx_status stage_tables(const qfx_plan* p, void* dst, void* stream, DeviceTables* out);
DeviceTables tables_at(void* base, const size_t offs[kTableRegions]);
// fold-adjoint partial entries of one site (the adjoint's per-site partial offsets)
int64_t adjoint_site_partials(const qfx_plan* p, const FoldSite& fs);

// contraction-tree planning (plan_tree.cpp)
bool tree_cut_search(const std::vector<std::vector<int>>& site_legs, int n_edges,
                     std::vector<int64_t>& edim, std::vector<int>& cut_edges, uint64_t cap_elems,
                     const std::vector<int64_t>& full, int* base_out, std::string* err);
bool build_tree_nodes(const std::vector<std::vector<int>>& site_legs, const std::vector<int64_t>& edim,
                      int base, const std::vector<uint64_t>& site_off, uint64_t arena_base,
                      std::vector<TreeNode>& nodes, uint64_t* arena_bytes,
                      std::vector<int>* root_legs, int64_t* max_el, std::string* err);

// the executor behind qfx_amplitudes (argument checks, items in flight, run)
qfx_status check_amplitudes_args(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                 int64_t slice_begin, int64_t slice_end, const void* out);
int64_t items_in_flight(const qfx_plan* p, size_t ws_bytes);
qfx_status exec_amplitudes(const qfx_plan* p, const DeviceTables& t, const uint64_t* x1,
                           int64_t n_batch, int64_t slice_begin, int64_t slice_end,
                           void* workspace, int64_t G, double* out, void* stream);

// profiling hooks
bool profile_on();
void profile_begin(void* stream, int* slot);
void profile_end(void* stream, int slot, int step, int variant, int kind, double flops,
                 double bytes);

void count_launch(int n = 1);

}  // namespace qfx
