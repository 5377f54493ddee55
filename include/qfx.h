/*
 * qfx.h -- C ABI of libqfx: tensor-network amplitudes of random quantum circuits on a
 * 2D qubit grid, computed on one GB300 GPU (sm_103a).
 *
 * What the library computes (arXiv:1905.00444):
 *   amp(x) = <x| C |0^n>, the quantity behind "Probability(circuit, s)" of the RCS
 *   benchmark (Fig. 1), for batches of bitstrings x = x1 u x2 that share x1 (fast
 *   sampling, Sec. III.B), as a sum over independent slices of the network (cuts,
 *   Sec. III.A).  The circuit is folded in time into one tensor per grid site (Sec. III,
 *   Fig. 3), each diagonal two-qubit gate becoming a bond of dimension 2 between the two
 *   sites; the sites are then contracted one by one, each contraction a complex GEMM in
 *   the TTGT form of Sec. III.E, with counted work F = 8 sqrt(v0 v1 v2) (Eq. 1).
 *
 * Conventions
 *   - qubit q = r * cols + c.  A bitstring of n qubits is ceil(n / 64) uint64 words (the
 *     plan's x1_words; one word up to 64 qubits): qubit q is bit q % 64 of word q / 64.
 *     Grids hold up to 144 qubits.
 *   - complex numbers are (re, im) pairs; complex64 = 2 x float, complex128 = 2 x double.
 *   - Every call returns a qfx_status.  On failure, qfx_last_error() (thread-local) holds
 *     a message.  No exception crosses the ABI and nothing aborts the process.
 *   - Host objects (qfx_circuit, qfx_plan) are opaque, owned by the library, created by
 *     *_create and freed by *_destroy.  They are immutable after creation and may be
 *     shared between threads.  A plan holds a host image of its tables (fold program,
 *     gate matrices, cuts, output order; a few hundred KB at most for the paper's
 *     shapes); the first compute call with a plan page-locks that image (under a lock;
 *     qfx_plan_upload does it explicitly).
 *   - All device buffers (inputs, outputs, workspace) are owned by the caller.  The
 *     compute entry points allocate no device memory: every call copies the plan's table
 *     image into the first bytes of the caller's workspace (an asynchronous copy on the
 *     call's stream) and keeps all other scratch there too.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = legacy stream).
 */
#ifndef QFX_H
#define QFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QFX_OK = 0,
  QFX_EINVAL = 1,       /* bad argument, bad circuit, bad plan option */
  QFX_ENOMEM = 2,       /* caller's workspace smaller than one work item needs */
  QFX_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  QFX_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
  QFX_EUNSUPPORTED = 5, /* valid request this build does not implement */
  QFX_EPLAN = 6         /* no plan meets the memory cap */
} qfx_status;

typedef enum {
  QFX_GATE_H = 0,
  QFX_GATE_SQRT_X = 1,
  QFX_GATE_SQRT_Y = 2,
  QFX_GATE_T = 3,
  QFX_GATE_CZ = 4,
  QFX_GATE_U1 = 5,  /* any single-qubit 2x2 matrix */
  QFX_GATE_U2 = 6,  /* any diagonal two-qubit gate */
  QFX_GATE_U4 = 7   /* any two-qubit 4x4 matrix (fSim, iSWAP, CNOT, ...) */
} qfx_gate_kind;

/* One gate.  For single-qubit gates `kind` is a label only; for two-qubit gates it selects
 * the form of `mat` (H .. U1 single-qubit, CZ and U2 diagonal, U4 general).
 *   single-qubit (q1 == -1): mat[0..7] = 2x2 complex, row-major, (re, im) interleaved:
 *                            mat[2*(2*row + col)] + i*mat[2*(2*row + col) + 1].
 *   CZ, U2 (q1 >= 0):        a diagonal gate; mat[0..7] = its 4 diagonal entries
 *                            d[2*b0 + b1] (b0 = value of q0, b1 = value of q1), interleaved.
 *                            Each such gate adds one bit (a leg of dimension 2) to its bond.
 *   U4 (q1 >= 0):            mat[0..31] = 4x4 complex G[2*o0 + o1][2*i0 + i1], row-major,
 *                            interleaved (o = output, i = input values of q0 and q1).  It is
 *                            split exactly as G = sum_k E_k (x) B_k, k = 2*o0 + i0, with
 *                            E_k = |o0><i0| on q0 and B_k[o1][i1] = G[2*o0 + o1][2*i0 + i1] on
 *                            q1: one leg of dimension 4 (two bits) on its bond.
 * The entries a kind does not use are ignored.  q0 and q1 must be grid neighbours.
 * Gates of one layer must act on disjoint qubits; layers run in increasing order.  A bond
 * holds at most 40 bits; its index reads the earliest gate's leg as the most significant
 * bits.  Entries must be finite.  The time fold computes in float-float arithmetic (FP32
 * pairs, about 48 significant bits, the FP32 exponent range), so the partial products of a
 * site's time line must stay within about 1e-30 .. 1e38 in magnitude; unitary gates and
 * the diagonal and projector pieces of two-qubit gates keep them at most 1. */
typedef struct {
  int32_t layer;
  int32_t q0;
  int32_t q1;
  int32_t kind;
  double mat[32];
} qfx_gate;

typedef struct qfx_circuit qfx_circuit;
typedef struct qfx_plan qfx_plan;

/* Sec. III (RQC class on a planar grid; Table I's "1+d+1" circuits).
 * Validates and copies the gate list (a1): qubit ranges, two-qubit gates only between
 * grid neighbours, disjoint qubits within a layer, layers >= 0, rows*cols <= 144.
 * Errors: QFX_EINVAL with the offending gate index in qfx_last_error(). */
qfx_status qfx_circuit_create(int32_t rows, int32_t cols, const qfx_gate* gates,
                              int64_t n_gates, qfx_circuit** out);

/* Same, from text: first line "grid R C", then one gate per line
 * "layer KIND q0 [q1] v0 v1 ... " with the gate's matrix values written out: 8 for every
 * kind but U4, 32 for U4 (KIND one of H SQRT_X SQRT_Y T CZ U1 U2 U4; q1 present only for
 * CZ, U2 and U4).
 * '#' starts a comment.  Errors: QFX_EINVAL with the line number. */
qfx_status qfx_circuit_from_text(const char* text, qfx_circuit** out);

void qfx_circuit_destroy(qfx_circuit* c);

typedef enum {
  QFX_PREC_FP32_SIMT = 0,   /* complex FP32 on the FMA pipes, 4 real FMAs per complex MAC */
  /* Split-precision modes on tcgen05 with FP32 accumulation.  The complex product is formed
   * from 4 real products (4M; the C3M names are the modes' family names), each the sum of
   * the term products above the mode's precision: */
  QFX_PREC_C3M_BF16X3 = 1,  /* 3 BF16 terms h, m, l; 6 term products; ~FP32 error */
  QFX_PREC_C3M_TF32X3 = 2,  /* 2 TF32 terms; 3 term products; ~2^-21 */
  QFX_PREC_C3M_BF16X2 = 3   /* 2 BF16 terms h, m; 3 term products (hm, mh, hh); ~2^-16, fastest */
} qfx_precision;

/* A cut (Sec. III.A): the bond between grid neighbours qa and qb is sliced into pieces
 * of `size` consecutive bond values (size a power of two dividing the bond dimension;
 * size 1 fixes the bond completely).  A bond's index reads the leg of its earliest
 * two-qubit gate as the most significant bit. */
typedef struct {
  int32_t qa;
  int32_t qb;
  int32_t size;
} qfx_cut;

typedef struct {
  uint64_t max_intermediate_bytes; /* cap on the largest intermediate tensor (complex64); 0 = none */
  const int32_t* open_sites;       /* x2 qubits (Sec. III.B), or NULL to let the planner take
                                      the last n_open sites of its contraction order */
  int32_t n_open;                  /* number of x2 qubits (<= 24); output index bit i = open site i */
  const qfx_cut* forced_cuts;      /* cuts always applied, first and in this order; cuts the
                                      cap needs come after them, and may narrow a forced
                                      one further (qfx_plan_cut reports the final sizes) */
  int32_t n_forced_cuts;
  int32_t precision;               /* qfx_precision */
  int32_t plan_family;             /* 0 = line sweep, 1 = contraction tree (see qfx_plan_create) */
  int32_t tc_flags;                /* tensor-core options, QFX_TC_* bits; 0 = default */
  const char* autotune_cache;      /* JSON file written by qfx_autotune, or NULL */
  uint64_t adjoint_store_bytes;    /* qfx_amplitudes_backward keeps the output of every step
                                      when they fit in this many bytes (0 = 4 GiB), else one
                                      boundary per grid line; 1 = always the latter */
} qfx_plan_opts;

/* Tensor-core accumulation.  Default: each complex tile is 128 x 128 with four TMEM
 * accumulators -- the hi x hi term products in "main" ones, all cross-term products in
 * "small" ones -- so the large accumulators see two additions per k-step (the tensor
 * core's FP32 accumulation loses a little at each addition).  QFX_TC_FAST_ACCUMULATION:
 * 128 x 256 tiles with one accumulator pair (fewer shared-memory reads, larger error). */
#define QFX_TC_FAST_ACCUMULATION 1
/* Default tiles stage the FP32 rows of B by tensor-map copies when the shape allows it
 * (Sd even and Sd a multiple or a divisor of 128, 16-byte aligned buffers).
 * QFX_TC_REGISTER_ROWS loads them with per-thread loads instead (same arithmetic). */
#define QFX_TC_REGISTER_ROWS 4

/* Sec. III.D (contraction order and cuts), Sec. III.A (slices), Sec. III.B (x2), Eq. 1.
 * Host only.  Plan family 1 (the region plans of Sec. III, Fig. 3): a contraction tree
 * built greedily -- contract the connected pair whose result grows least over its larger
 * operand -- with cuts chosen by halving, one at a time, the bond of the largest
 * intermediate that lowers the largest intermediate most, until it fits the cap.  Each
 * node is a TTGT step (permutes where the operands' shared legs are not in place, then the
 * step GEMM below with P, Sd the larger operand's legs before and after the shared ones).
 * Contractions longer than 1024 are summed in chunks of 1024, each added into the result.
 * Split precisions run every node the tensor-core tiles take on them (as for the line
 * sweep).  qfx_amplitudes, qfx_amplitudes_static and batches run tree plans (the adjoint
 * and the autotune cache do not: QFX_EUNSUPPORTED, ignored).
 * Plan family 0: the plan sweeps the grid line by line (along the shorter grid dimension),
 * absorbing one site per step so that every step is a strided batched complex GEMM
 * C[nh][p][nl][s] = sum_k S[k][nh*NL+nl] * B[p][k][s] with no tensor transpose; then it
 * adds cuts (greedily halving the bond that keeps the total work lowest) until the
 * largest intermediate fits the cap.
 * Errors: QFX_EINVAL (bad options), QFX_EPLAN (cap cannot be met, largest tensor above
 * 2^50 elements, or a bond that keeps more than 2^30 values after its cuts). */
qfx_status qfx_plan_create(const qfx_circuit* c, const qfx_plan_opts* opts, qfx_plan** out);
void qfx_plan_destroy(qfx_plan* p);

typedef struct {
  int64_t n_slices;            /* product of the cut radices */
  int32_t n_steps;             /* line sweep: sites absorbed, = number of qubits (step 0 is
                                  free); contraction tree: its n - 1 pairwise contractions */
  int32_t n_open;
  int32_t n_cuts;
  int32_t n_sites;
  double flops_per_item;       /* Eq. 1 flops of one (slice, x1) work item */
  double bytes_per_item;       /* algorithmic bytes: each GEMM operand read once, output written once */
  int64_t max_elements;        /* largest intermediate, complex64 elements */
  uint64_t item_bytes;         /* workspace one work item needs */
  uint64_t workspace_min;      /* workspace for one item plus the shared header */
  int32_t largest_step;        /* index of the step with the most flops */
  int32_t precision;
  int32_t x1_words;            /* uint64 words per bitstring, ceil(n / 64) */
} qfx_plan_stats;

qfx_status qfx_plan_info(const qfx_plan* p, qfx_plan_stats* out);

/* Workspace bytes for `n_concurrent` work items in flight at once. */
uint64_t qfx_workspace_bytes(const qfx_plan* p, int64_t n_concurrent);

typedef struct {
  int32_t site;       /* line sweep: qubit absorbed by this step; contraction tree: id of
                         the node's result (the sites are tensors 0 .. n-1, node results
                         n, n+1, ... in step order) */
  int32_t variant;    /* kernel tile variant chosen for it */
  int64_t P, K, N, NL, Sd;  /* shapes as in qfx_plan_create's formula; NH = N / NL */
  double flops;       /* 8*P*K*N*Sd = 8 sqrt(v0 v1 v2), Eq. 1 */
  double bytes;       /* 8*(P*K*Sd + K*N + P*N*Sd) */
  int32_t parts;      /* contraction-tree nodes: > 0 when K runs as this many 1024-long chunks
                         side by side (partial products summed in FP64), else 0 */
  int32_t reserved;
} qfx_step_info;

qfx_status qfx_plan_step(const qfx_plan* p, int32_t i, qfx_step_info* out);
qfx_status qfx_plan_cut(const qfx_plan* p, int32_t i, qfx_cut* out);
/* The plan's x2 qubits, in output-bit order (out must hold n_open entries). */
qfx_status qfx_plan_open_sites(const qfx_plan* p, int32_t* out);

/* Page-locks the plan's host table image so that the copy every compute call makes from
 * it is asynchronous and can be recorded into a CUDA graph.  The first compute call with
 * the plan does this implicitly; make that call, or this one, before any stream capture.
 * If the system refuses to page-lock the image, it stays pageable (the copies stay
 * correct but may make the host wait for the stream).  Allocates no device memory. */
qfx_status qfx_plan_upload(const qfx_plan* p);

/* Amplitudes (Sec. III.A-III.B; the sum over paths of Sec. III.A and III.C).
 *   x1        device, [n_batch][x1_words] uint64 bitstrings (x1_words = ceil(n / 64) from
 *             qfx_plan_info, 1 up to 64 qubits); the bits of the open sites are ignored.
 *   slices    [slice_begin, slice_end) of the plan's n_slices; a sub-range gives that
 *             range's contribution (sharding, or a fraction of paths).
 *   workspace device, ws_bytes >= qfx_plan_stats.workspace_min, 256-byte aligned; more
 *             workspace lets more (slice, x1) items run concurrently.  Its first bytes
 *             receive the plan's tables (copied on `stream` by every call), the rest the
 *             per-item headers, boundary tensors and site tensors.
 *   out       device complex128 [n_batch][2^n_open], overwritten with
 *             2^(sum of per-site scale exponents) * sum over slices (in slice order, FP64).
 * Asynchronous on `stream`.  Errors: QFX_EINVAL, QFX_ENOMEM, QFX_ECUDA. */
qfx_status qfx_amplitudes(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                          int64_t slice_begin, int64_t slice_end, void* workspace,
                          size_t ws_bytes, double* out, void* stream);

/* Size of the scratch array compiled into the library for qfx_amplitudes_static. */
#define QFX_STATIC_SCRATCH_BYTES (64ull << 20)

/* qfx_amplitudes without a caller workspace, for callers that cannot allocate device
 * memory (a host application whose memory manager owns the device, code that cannot
 * afford cudaMalloc's implicit synchronisation, a plugin handed only its buffers).
 * The paper has no counterpart: it is an interface convenience of this library.
 *   Same arguments and results as qfx_amplitudes, minus the workspace: scratch is a
 *   file-scope device array of QFX_STATIC_SCRATCH_BYTES (64 MiB) that every GPU loading
 *   the library holds until exit.  The plan's tables plus qfx_workspace_bytes(p, 1) must
 *   fit in it, else QFX_ENOMEM with both sizes in the message.
 *   Allocates nothing.  The first call on a device looks up the array's device address
 *   (make it before any stream capture).  All calls share the array: calls that overlap
 *   on the GPU race, and each call rewrites what it reads.  The plan's tables are copied
 *   into the array from the plan's own host image; this entry point does not page-lock
 *   that image, so unless qfx_plan_upload or another call has, the copy is from pageable
 *   memory and may make the host wait for work already queued on the stream. */
qfx_status qfx_amplitudes_static(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                 int64_t slice_begin, int64_t slice_end, double* out,
                                 void* stream);

/* Batched execution (Sec. III.A: slices are independent paths; Sec. III.B: x1 batches).
 * Many work items -- every (slice, x1) of every listed item, of any mix of plans and
 * shapes -- run together:
 * - items whose steps all run FP32 tiles (FP32 plans, and split-precision plans whose
 *   step shapes the tensor-core tile does not take) and whose largest step has fewer
 *   than 512 output tiles: in ONE persistent kernel, a device task queue of fold chunks,
 *   scale chunks, contraction-step tiles (each step's plan-chosen variant) and FP64
 *   accumulations, with per-segment completion counters as dependencies and bounded
 *   waits;
 * - items with tensor-core steps, larger items and contraction trees: as ONE CUDA graph
 *   built at prepare time, every item's launch sequence on one of up to 16 parallel
 *   lanes, each lane with its own workspace slot (`slots` = lanes); the persistent
 *   launch of the small items, if any, is a node of the same graph.
 * Each batch item's `out` rows get the same values qfx_amplitudes would produce. */
typedef struct {
  const qfx_plan* plan;
  const uint64_t* x1;      /* device [n_batch][x1_words] */
  int64_t n_batch;
  int64_t slice_begin, slice_end;
  double* out;             /* device complex128 [n_batch][2^n_open], overwritten */
} qfx_batch_item;

typedef struct qfx_batch qfx_batch;

/* Workspace that lets `slots` work items be in flight at once (an upper bound). */
uint64_t qfx_batch_workspace_bytes(const qfx_batch_item* items, int32_t n_items, int64_t slots);

/* Builds the schedule and uploads it into `workspace` (synchronously on `stream`),
 * together with one copy of each distinct plan's tables at the workspace's start.  The
 * workspace, items' x1 and out buffers must stay valid while
 * the batch is used.  Errors: QFX_EINVAL, QFX_ENOMEM, QFX_ECUDA. */
qfx_status qfx_batch_prepare(const qfx_batch_item* items, int32_t n_items, void* workspace,
                             size_t ws_bytes, qfx_batch** out, void* stream);

/* Clears the queue counters and launches the persistent kernel (or launches the batch's
 * graph): asynchronous, no allocation and no host synchronisation, so it can itself be
 * captured in a CUDA graph.  A dependency wait that expires (5 s) is reported by qfx_sync
 * as QFX_ETIMEOUT. */
qfx_status qfx_batch_run(const qfx_batch* b, void* stream);

qfx_status qfx_batch_info(const qfx_batch* b, int64_t* n_work, int64_t* n_tasks, int64_t* slots);
void qfx_batch_destroy(qfx_batch* b);

/* Adjoint (not in the paper; the multilinear structure of Sec. III's network makes it
 * exact): gradients of a real loss L(amp) with respect to every gate's 8 matrix values.
 *   grad_out   device complex128 [n_batch][2^n_open]: dL/dRe(amp) + i dL/dIm(amp) for the
 *              amplitudes qfx_amplitudes returns for the same arguments (PyTorch's
 *              convention; for L = sum |amp|^2 it is 2 amp).
 *   grad_gates device complex128 [n_gates][4], overwritten: for gate g of the caller's
 *              list, dL/dRe + i dL/dIm of its mat entries (2x2 row-major, or the 4
 *              diagonal entries of a two-qubit gate), summed over batch and slices.
 *   workspace  device, >= qfx_backward_workspace_bytes(p), 256-byte aligned.
 * Runs the contraction in FP32 on the FMA path.  The forward sweep keeps every step's
 * output when they fit in the plan's adjoint_store_bytes; otherwise it keeps the boundary
 * at each line start and the reverse sweep recomputes one line at a time.  Errors: QFX_EINVAL, QFX_ENOMEM, QFX_ECUDA,
 * QFX_EUNSUPPORTED (more than 64 time-line event slots on one site -- a U4 gate's q1
 * event takes 4 -- or a U4 gate: its 16 entries do not fit the 4 per gate of grad_gates;
 * qfx_amplitudes_backward_full takes them). */
qfx_status qfx_amplitudes_backward(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                   int64_t slice_begin, int64_t slice_end, const double* grad_out,
                                   double* grad_gates, void* workspace, size_t ws_bytes,
                                   void* stream);

/* Same, for circuits with any gate kinds: grad_gates is device complex128 [n_gates][16],
 * overwritten; entry j of gate g is the gradient with respect to the j-th complex value
 * of its mat (a U4 gate's 16 entries G[r][c] at j = 4*r + c; other gates their 4 values,
 * then zeros).  For a U4 gate G[2*o0 + o1][2*i0 + i1] is entry (o1, i1) of the block
 * B_k, k = 2*o0 + i0, that its q1 event applies, so its gradient is that block's.  Same
 * workspace and errors (without the U4 restriction). */
qfx_status qfx_amplitudes_backward_full(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                                        int64_t slice_begin, int64_t slice_end,
                                        const double* grad_out, double* grad_gates,
                                        void* workspace, size_t ws_bytes, void* stream);
uint64_t qfx_backward_workspace_bytes(const qfx_plan* p);

/* Autotuner: times every compatible FP32 tile variant of each distinct step shape of `p`
 * (on `workspace`, shrinking the problem to fit it) and records the fastest per shape
 * (N, K, NL, Sd) in the JSON file `cache_path` (existing entries are kept and not
 * re-timed).  Plans created with opts.autotune_cache use the recorded variants.
 * Synchronises `stream`.  Errors: QFX_EINVAL, QFX_ENOMEM, QFX_ECUDA. */
qfx_status qfx_autotune(const qfx_plan* p, const char* cache_path, void* workspace,
                        size_t ws_bytes, void* stream);

/* Waits for `stream` and reports any asynchronous CUDA error as QFX_ECUDA, and a
 * tensor-core kernel that gave up a bounded wait (about 1 s) as QFX_ETIMEOUT. */
qfx_status qfx_sync(void* stream);

/* Measured tensor-core peak of a precision's operand kind (BF16 for the BF16 modes, TF32
 * for TF32x3): one CTA per SM issues `mmas_per_sm` (>= 256, rounded up to a multiple of
 * 256) back-to-back tcgen05.mma of M = 128, N = 256 and one K step from shared memory
 * into TMEM; `*tflops` = dense flop/s of that kind (2 M N K per MMA) over the timed launch.
 * Runs one warm-up launch and one timed launch on `stream` and synchronises.  Errors:
 * QFX_EINVAL, QFX_ECUDA, QFX_ETIMEOUT. */
qfx_status qfx_tensor_peak(int32_t precision, int64_t mmas_per_sm, double* tflops, void* stream);

/* One contraction step of the TTGT form (Sec. III.E), for tests and microbenchmarks:
 * C[nh][p][nl][s] = sum_k S[k][nh*NL + nl] * B[p][k][s], complex64, all device pointers,
 * 16-byte aligned, no aliasing.  `variant` < 0 lets the library choose (FP32 only);
 * FP32 tile variants are 0-9 (0-4 need an even Sd) and their fill variants 20-23 (even
 * Sd) and 25-28, which compute 4096 or 2048 outputs per CTA for grids that would leave SMs
 * idle; every variant gives bit-identical results.
 * Tensor-core precisions run on tcgen05 when N % 16 == 0 and N <= 128 or a multiple of 128
 * (fast accumulation: N <= 256 or a multiple of 256), K a multiple of the term's k step
 * (16 for BF16x3 and BF16x2, 8 for TF32x3) and P*Sd >= 128, otherwise on the FP32
 * path; they need `scratch` of qfx_step_scratch_bytes(K, N, precision) bytes, 256-byte
 * aligned (NULL is fine for FP32).  Variant 12 selects fast accumulation (see
 * QFX_TC_FAST_ACCUMULATION) for a tensor-core step; variant 13 keeps the default tile but
 * loads the FP32 rows of B with per-thread loads instead of tensor-map copies (same
 * arithmetic, for comparison).  Test hook: variant 99 with a tensor-core step
 * withholds the stream of S, so every CTA's bounded waits expire (about 1 s each, run
 * it on at most a few hundred columns); qfx_sync then reports QFX_ETIMEOUT and the
 * context stays usable.  Errors: QFX_EINVAL, QFX_ENOMEM (scratch), QFX_ECUDA. */
qfx_status qfx_contract_step(const void* S, const void* B, void* C, int64_t P, int64_t K,
                             int64_t N, int64_t NL, int64_t Sd, int32_t precision,
                             int32_t variant, void* scratch, size_t scratch_bytes,
                             void* stream);

/* Scratch bytes a tensor-core step with these K and N needs (0 for FP32). */
uint64_t qfx_step_scratch_bytes(int64_t K, int64_t N, int32_t precision);

/* Tensor transpose (Sec. III.E): out = in with axes reordered; complex64, rank <= 10.
 * shape[] is the input shape (C order); out axis a is input axis perm[a].
 * Device pointers, no aliasing.  Errors: QFX_EINVAL for a bad permutation or rank. */
qfx_status qfx_permute(const void* in, void* out, int32_t rank, const int64_t* shape,
                       const int32_t* perm, void* stream);

/* Fast sampling with frugal rejection (Sec. III.B): one sample per x1 batch.
 *   x1         device uint64 [n_batch][x1_words], the batches' x1 (as passed to qfx_amplitudes).
 *   amps       device complex128 [n_batch][2^n_open], 16-byte aligned: qfx_amplitudes'
 *              output for the same plan and x1 (any slice range: a fraction f of the
 *              slices gives noisy sampling at fidelity about f, Sec. III.C).
 *   u          device float64 [n_batch][2^n_open]: uniform variates in [0, 1), u[b][t] for
 *              scan position t of batch b.
 *   scan_mask  device uint64 [n_batch]: batch b examines x2 = t XOR scan_mask[b] (low
 *              n_open bits used), t = 0, 1, ...
 *   M          rejection constant (> 0): candidate t is accepted when
 *              u[b][t] < 2^n |amp|^2 / M, evaluated in FP64 as p = re*re + im*im, then
 *              p * (2^n / M), each operation rounded to nearest (no fused multiply-add).
 *              With amplitudes of fidelity f pass M * f.
 *   x2_out     device int64 [n_batch]: the first accepted x2 in scan order, -1 if none.
 *   bits_out   device uint64 [n_batch][x1_words] or NULL: x1 with the bit of open_sites[i]
 *              set to bit i of x2 (x1 unchanged where x2_out is -1).
 * One block per batch; asynchronous on `stream`; no allocation.
 * Errors: QFX_EINVAL (NULL or misaligned pointers, M not finite and > 0), QFX_ECUDA. */
qfx_status qfx_frugal_select(const qfx_plan* p, const uint64_t* x1, int64_t n_batch,
                             const double* amps, const double* u, const uint64_t* scan_mask,
                             double M, int64_t* x2_out, uint64_t* bits_out, void* stream);

/* Kernel timing for measurement (not needed for computing): while enabled, each
 * contraction-step launch is bracketed by CUDA events on its own stream. */
typedef struct {
  int32_t step;       /* plan step index, or -1 for qfx_contract_step */
  int32_t variant;
  int32_t kind;       /* 0 = contraction step, 1 = fold, 2 = scale, 3 = accumulate,
                         4 = permute, 5 = frugal select */
  float ms;
  double flops;
  double bytes;
} qfx_kernel_time;

qfx_status qfx_profile_enable(int32_t on);
/* Waits for the recorded events; copies up to `max` records; returns the count in *n
 * and clears the record list. */
qfx_status qfx_profile_collect(qfx_kernel_time* out, int32_t max, int32_t* n);

/* Test hooks (not needed for computing).  Each makes one bounded device wait run out on
 * purpose, so that the error path -- the waiting kernel records QFX_ETIMEOUT in its status
 * word, every CTA returns, the context stays usable -- can be tested without faulting or
 * hanging the GPU.  The paper has no counterpart.
 *   qfx_debug_permute_withhold: the calling thread's next qfx_permute that takes the
 *     tensor-map path issues none of its copies and waits at most wait_ns (1e3..1e9) for
 *     them; the output is left unwritten and qfx_sync reports QFX_ETIMEOUT.
 *   qfx_debug_batch_stall: one dependency of a persistent-kernel batch's schedule is made
 *     unreachable and every dependency wait is limited to wait_ns (1e3..5e9); the next
 *     qfx_batch_run gives up after wait_ns and qfx_sync reports QFX_ETIMEOUT.  The batch
 *     is broken for good (destroy it).  QFX_EUNSUPPORTED for graph batches.
 * Errors: QFX_EINVAL (bad argument), QFX_ECUDA. */
qfx_status qfx_debug_permute_withhold(int64_t wait_ns);
qfx_status qfx_debug_batch_stall(qfx_batch* b, int64_t wait_ns);

/* Number of kernels this library has launched since it was loaded. */
uint64_t qfx_launch_count(void);

const char* qfx_last_error(void);
const char* qfx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QFX_H */
