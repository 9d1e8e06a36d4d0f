/*
 * dls.h -- C ABI of the GB300 (sm_103a) Discontinuous DLS block compressor.
 *
 * Method: arXiv 2601.20113, "A Data-Informed Local Subspaces Method for
 * Error-Bounded Lossy Compression of Large-Scale Scientific Datasets".
 * The field is partitioned into independent space-time blocks (patches,
 * Algorithm 1 step 2); each block gets its own basis from the right singular
 * vectors of its data matrix, computed the cross-product way (Gram matrix +
 * symmetric eigensolve; Sec. 2.3 Eq. 2-3, Sec. 2.7.1); its coefficients are
 * the projection S = C^T P (Sec. 2.5, Eq. 5); the retained prefix is the
 * smallest one meeting the local L2 tolerance (Sec. 2.4 Eq. 4, Sec. 2.5
 * Eq. 6), found by bisection; coefficients are quantized (in place of
 * bit-grooming) and, for pointwise bounds, a correction pass makes every
 * point meet the bound.  Streams follow Sec. 2.7.2: an addressable header,
 * an offset table from an exclusive scan of record sizes, packed records.
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers, h_* are host pointers.  The
 *     caller owns every buffer; the library keeps only small cached state
 *     (pinned status words, the rank model, graph and tuning caches).
 *   - Calls are ordered on `stream` and asynchronous, except that values the
 *     call returns through host pointers (out_bytes, reports) are written
 *     before it returns: such calls synchronize `stream` once.
 *   - Return value: DLS_OK (0) or a negative DLS_ERR_* status.  On error, the
 *     contents of output buffers are unspecified.
 *   - Fields hold nvars variables back to back, each laid out
 *     [nt][nz][ny][nx] (x fastest), in float32 or float64.
 */
#ifndef DLS_H
#define DLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* dls_stream_t;

enum { DLS_F32 = 0, DLS_F64 = 1 };
/* Bound types.  ABS: absolute pointwise bound.  REL_RANGE: bound = value x
 * (max - min) of each variable (one extra read of the field).  NRMSE: the
 * paper's global L2 target in percent, eps = eps_t ||u|| / 100 (Sec. 2.4);
 * no pointwise correction in that mode. */
enum { DLS_EB_ABS = 0, DLS_EB_REL_RANGE = 1, DLS_EB_NRMSE = 2 };
/* Arithmetic of the Gram and projection products.
 *   FP64:   double precision everywhere (the plain form).
 *   FP32:   FP32 products on the CUDA cores with FP32 accumulation; FP32
 *           Jacobi eigensolve, its eigenvectors orthonormalised in FP64 (to
 *           below the rounding of the stored modes); every stored decision
 *           (quantized coefficient, rank test, correction, escape) keeps FP64
 *           semantics.
 *   TF32X3: as FP32, with the block Gram on the tensor cores (tcgen05,
 *           kind::tf32) as a 3-term TF32 split product (hi hi + hi lo + lo hi,
 *           FP32 accumulation; about 21 bits of each value) for
 *           16 x 16 x bz x 16 blocks of a field whose x extent is a multiple
 *           of 4; other blocks use the FP32 Gram.
 *   TF32:   as TF32X3 with the one product hi hi (10-bit mantissas).
 *   BF16X3: as TF32X3 with the Gram as the three-product BF16 split of
 *           Henry, Tang and Heinecke (2019) on tcgen05 kind::f16:
 *           b0 b0 + b0 b1 + b1 b0 with b0 = bf16(x), b1 = bf16(x - b0)
 *           (relative error about 2^-16).
 *   BF16:   as BF16X3 with the one product b0 b0 (8-bit mantissas).
 * In every non-FP64 mode the projection, the quantizer, the rank test and
 * the corrections are those of FP32 (CUDA cores, FP64-semantics decisions):
 * the modes differ in the Gram, and so in the basis, only.  Non-FP64 modes
 * apply to float32 fields with a Gram order <= 16; other fields take the
 * FP64 form whatever the mode. */
enum { DLS_PREC_FP64 = 0, DLS_PREC_TF32X3 = 1, DLS_PREC_BF16X3 = 2, DLS_PREC_FP32 = 3, DLS_PREC_TF32 = 4,
       DLS_PREC_BF16 = 5 };
/* Rank selection.  SEARCH: bisection of Algorithm 1.  LEARNED: the loaded
 * block-rank MLP (dls_set_rank_model) predicts the rank r; it is accepted
 * only if pass(r) holds and pass(r-1) does not (the smallest passing rank next
 * to the prediction), otherwise the bisection decides.  TAIL: as LEARNED with
 * the prediction taken from the eigenvalue tails, sum_{i>=r} lambda_i plus a
 * uniform quantization-noise estimate (a baseline without the network).
 * LEARNED and TAIL apply to the non-FP64 precision modes. */
enum { DLS_RANK_SEARCH = 0, DLS_RANK_LEARNED = 1, DLS_RANK_TAIL = 2 };

enum {
  DLS_OK = 0,
  DLS_ERR_INVALID_ARG = -1,   /* bad parameter, null pointer, bad size */
  DLS_ERR_CAPACITY = -2,      /* output too small; *out_bytes holds the size needed */
  DLS_ERR_NONFINITE = -3,     /* NaN or Inf in the input field */
  DLS_ERR_CORRUPT = -4,       /* stream fails structural validation */
  DLS_ERR_CUDA = -5,          /* a CUDA runtime call failed */
  DLS_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
  DLS_ERR_BOUND_VIOLATED = -7,/* dls_verify: some point exceeds its bound */
  DLS_ERR_WORKSPACE = -8,     /* workspace missing or smaller than dls_workspace_size */
  DLS_ERR_NO_MODEL = -9       /* LEARNED rank mode without a loaded model */
};

typedef struct {
  int32_t nvars;          /* >= 1, <= 64 */
  int64_t dims[4];        /* nx, ny, nz, nt (nz = 1 for 2-D fields) */
  int32_t block[4];       /* bx, by, bz, bt; 1 <= block[i] <= dims[i];
                             min(bx*by*bz, bt) <= 32; bx*by*bz*bt <= 2^26 */
  int32_t dtype;          /* DLS_F32 / DLS_F64 */
  int32_t eb_type;        /* DLS_EB_* */
  const double* eb;       /* host array of nvars values, each > 0 */
  int32_t rank_cap;       /* >= 0; per block min(rank_cap, Gram order) */
  int32_t precision;      /* DLS_PREC_* */
  int32_t rank_mode;      /* DLS_RANK_* */
  int64_t block_begin;    /* compress blocks [block_begin, block_end) only; */
  int64_t block_end;      /* block_end < 0 means through the last block      */
  /* Fixed basis (Sec. 4: data-adaptive SVD modes against fixed cosine or
   * random modes).  Null: every block uses its own eigenvectors (the method).
   * Otherwise a host array of basis_n x basis_n doubles, basis[a * basis_n + k]
   * = component a of mode k, the columns orthonormal to 1e-12: blocks whose
   * Gram order equals basis_n project on these modes, in the given order,
   * instead of their own; other blocks are unchanged.  Requires
   * DLS_PREC_FP64 and DLS_RANK_SEARCH (else DLS_ERR_INVALID_ARG), as does a
   * basis_n outside [1, 32] or a basis that is not orthonormal.  Every record
   * stores its modes, so decompression needs nothing more.  dls_compress
   * copies the array on each call (it may be freed on return); a plan copies
   * it once, at dls_plan_create, into its workspace. */
  const double* basis;
  int32_t basis_n;
  /* Statistics of the whole field, for a call that compresses one part of it
   * (a rank's z-slab; Sec. 2.7.1 data distribution).  Null: the field passed
   * is the whole field.  Otherwise a host array of nvars x 4 doubles, per
   * variable {min, max, sum of squares, number of points} of the whole field
   * (an all-reduce of the parts' own statistics): REL_RANGE takes the range,
   * NRMSE the norm and the point count (Sec. 2.4 Eq. 4: eps and the points K
   * of eps_l^2 = eps^2 N / K) from it instead of from the part, so that every
   * part resolves the same bound and the parts' records are those of the
   * whole field.  Points must be >= 1 and equal across variables, min <= max,
   * the sum >= 0, all finite, the count integral (else DLS_ERR_INVALID_ARG).  Copied on each call
   * (plans: once, at dls_plan_create). */
  const double* global_stats;
  /* Correction section codec (the lossless stage after the lossy map, Sec.
   * 2.5 and Algorithm 1 step 3; undone first in Sec. 2.6).  0: dense or
   * entry-list corrections only.  1: also the Rice-coded form (record flag 8)
   * wherever it is strictly smaller: the corrections in chunks of 1024
   * elements, each nonzero as the Rice code (parameter kr in [0, 20], the
   * fewest bits) of the zeros before it and zigzag(k) - 1 in wv bits, one more
   * code for the zeros to the chunk end; the section holds the word count,
   * kr | wv << 8, the chunks' bit offsets and the coded words.  Other values:
   * DLS_ERR_INVALID_ARG.  The decoder reads both. */
  int32_t corr_codec;
} dls_params;

/* Worst-case stream size for these parameters (each record is at most the
 * raw block plus 16 bytes).  0 if the parameters are invalid. */
size_t dls_compress_bound(const dls_params* p);

/* Device workspace dls_compress needs, in bytes (caller allocates, 256-byte
 * aligned).  0 if the parameters are invalid.  For a float32 field compressed
 * in a non-FP64 precision mode over its whole block range, whose x extent is
 * not a multiple of 4 (x lines not a multiple of 16 bytes) while block[0] is,
 * it includes a copy of the field with x lines padded to a multiple of 4
 * values: the staged kernels read their tiles by TMA from that copy, written
 * at the start of every compression. */
size_t dls_workspace_size(const dls_params* p);

/* Compress a device field (Algorithm 1, step 2-3; Sec. 2.7.2 stream).
 * d_in: nvars * nx*ny*nz*nt values of p->dtype.  d_out: out_cap bytes.
 * d_workspace: ws_bytes >= dls_workspace_size(p).  On success *out_bytes is
 * the stream size.  On DLS_ERR_CAPACITY *out_bytes is the size needed.
 * DLS_ERR_CORRUPT means a record failed the packer's own consistency check
 * (an internal fault, not an input error); the stream is then not valid.
 * Synchronizes `stream` once to read the stream size. */
int dls_compress(const dls_params* p, const void* d_in, void* d_out, size_t out_cap,
                 size_t* out_bytes, void* d_workspace, size_t ws_bytes, dls_stream_t stream);

/* Statistics of the field d_in (one part of a larger field, or all of it),
 * per variable {min, max, sum of squares, number of points} into h_stats
 * (host, nvars x 4 doubles), by the statistics pass a compression runs for
 * the relative and NRMSE bounds (Sec. 2.4): the sum of squares in the same
 * fixed order, so a single part's result given back as p->global_stats
 * resolves the bound the part resolves on its own.  A data-distributed
 * field (Sec. 2.7.1: each rank a z-slab) combines its parts' results --
 * min of mins, max of maxes, sums of the rest -- into the global_stats of
 * every part's compression.  p->global_stats is ignored here.  d_workspace
 * as for dls_compress.  DLS_ERR_NONFINITE if the part holds a NaN or an
 * infinity.  Synchronizes `stream`. */
int dls_field_stats(const dls_params* p, const void* d_in, double* h_stats, void* d_workspace, size_t ws_bytes,
                    dls_stream_t stream);

/* Reusable compression plan for fixed parameters and buffers (a time series
 * of snapshots written into the same buffers, for example).  Creation
 * validates like dls_compress, picks the occupancy form of the per-block
 * kernels for each shape class of the plan's blocks by timing both forms on
 * the real data (two full compressions per form, the classes timed apart by
 * events between their kernels; each class's choice is cached as a JSON line
 * in the file named by the environment variable DLS_AUTOTUNE_CACHE when set,
 * keyed by the parameters and the class; dls_plan_tuning reports it), then
 * captures the whole compression
 * (status reset, bound resolution, the persistent per-block kernel over every
 * block of every variable, scan + header, record placement and the deferred
 * record packer, status readback) in one CUDA graph.  Execution returns what
 * dls_compress returns.  Executing replays the graph and synchronizes `stream`.
 * The plan owns a small pinned status buffer; buffers stay owned by the
 * caller and must outlive the plan.  Creation writes d_out and d_workspace. */
typedef struct dls_plan dls_plan;
int dls_plan_create(const dls_params* p, const void* d_in, void* d_out, size_t out_cap, void* d_workspace,
                    size_t ws_bytes, dls_stream_t stream, dls_plan** out_plan);
int dls_plan_execute(dls_plan* plan, size_t* out_bytes, dls_stream_t stream);
/* Chosen occupancy form of the whole-block class (as dls_plan_tuning's
 * forms[0]) and the device ms of the per-block kernels, scan and packing of
 * one compression with every class in form 1 and in form 2 (0 if the choices
 * came from the cache or the form has one variant). */
int dls_plan_info(const dls_plan* plan, int32_t* variant, float* tune_ms);
/* The plan's occupancy form per shape class -- 1: the kernels built for fewer
 * CTAs per SM with more registers per thread (2 per SM for the staged kernels,
 * 1 for the space-side kernel), 2: built for more (4, 2) -- and the device time
 * that chose it.  Classes: [0] "whole", the blocks of the full block
 * shape that the encode kernel finishes at the predicted rank (Sec. 2.5 rank
 * step); [1] "rest", what the searching kernels take: edge blocks of smaller
 * shapes (Sec. 2.7.1 partition remainders), predictions the exact test
 * rejects, blocks whose Gram side is space, or every block when the plan
 * searches.  forms: 2 entries (form 1 or 2 of each class); class_ms: 4
 * entries, class_ms[2 c + f - 1] = ms of class c's kernels in form f during
 * tuning (0 if the choices came from the cache).  The forms run the same code,
 * so the stream does not depend on them.  Either pointer may be null. */
int dls_plan_tuning(const dls_plan* plan, int32_t* forms, float* class_ms);
/* Device time in ms of the per-block compression kernels during the most
 * recent dls_plan_execute (events recorded around them inside the graph; waits
 * for that execution), and the number of kernel nodes in the plan's graph.
 * Either pointer may be null. */
int dls_plan_timing(const dls_plan* plan, float* kernel_ms, int32_t* kernel_nodes);
/* Device time in ms of each stage of the most recent dls_plan_execute of a
 * mixed-precision plan (FP32 / TF32X3; zeros for the FP64 form and for plans
 * without time-side blocks), from events inside the graph (waits for that
 * execution): ms[0] the Gram pass (k_gram), ms[1] the eigensolve and rank
 * prediction (k_eig), ms[2] the Rayleigh-Ritz pass of the blocks that need it
 * (k_rrgram, k_eig), ms[3] the encode pass at the predicted rank with its
 * exact test and deferred records (k_enc), ms[4] the blocks left to the
 * searching kernel (k_tile, and k_mixed for blocks whose Gram side is space),
 * ms[5] the scan of record sizes and the record packing.  count >= 6
 * (further entries are set to 0). */
int dls_plan_phase_timing(const dls_plan* plan, float* ms, int32_t count);
/* Releases the plan's graph, events and pinned status buffer (not the
 * caller's buffers).  A null plan is accepted.  Call it once the last
 * execution has returned (dls_plan_execute synchronizes its stream). */
int dls_plan_destroy(dls_plan* plan);

/* Device staging bytes dls_compress_host needs: the input field, the stream
 * bound and the workspace, each 256-byte aligned.  0 if parameters are invalid. */
size_t dls_host_staging_size(const dls_params* p);

/* End-to-end compression of a HOST field (host in, host stream out): copies
 * h_in to the device, runs dls_compress, copies the stream back to h_out.
 * The stream equals dls_compress's.  For the FP32/TF32X3 forms with an
 * absolute bound, the field is copied one slab of block[3] time steps of one
 * variable at a time on an internal stream, each slab's blocks compressed as
 * soon as it has landed (so the copy hides most of the compression).
 * Pinned host memory (cudaHostAlloc) gives full copy bandwidth; pageable
 * memory works but is slower.  d_staging: staging_bytes >= dls_host_staging_size(p),
 * 256-byte aligned, owned by the caller.  out_cap bounds the host output.
 * Synchronizes `stream`; *out_bytes as in dls_compress. */
int dls_compress_host(const dls_params* p, const void* h_in, void* h_out, size_t out_cap, size_t* out_bytes,
                      void* d_staging, size_t staging_bytes, dls_stream_t stream);

/* Compression that allocates nothing (the paper has no counterpart: this is a
 * library convenience).  For callers that cannot allocate device memory when
 * they compress, e.g. an in-situ hook inside a simulation whose memory pools
 * already hold the whole device, or code running where CUDA allocation calls
 * are not allowed.  Same arguments and result as dls_compress, without the
 * workspace: the workspace is a 64 MiB device array inside this library.
 *   - Fields whose dls_workspace_size(p) exceeds 64 MiB are rejected with
 *     DLS_ERR_WORKSPACE (float32 blocks of 16^3 x 16 need about 8.2 bytes of
 *     workspace per point: up to roughly 8 million points; about 4 bytes more
 *     per point where the workspace holds the pitched copy of a field whose x
 *     extent is not a multiple of 4, see dls_workspace_size).
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     Under CUDA's lazy module loading (the default) that lookup is also when
 *     the array is placed in device memory, so the first call needs 64 MiB of
 *     free device memory: make it before the caller's pools take the device,
 *     or set CUDA_MODULE_LOADING=EAGER.  Later calls allocate nothing.
 *   - Invalid parameters return the status dls_compress returns for them.
 *   - Every call on a device shares the array: calls that overlap on the GPU
 *     (different streams or host threads) race and must be serialised by the
 *     caller.  Each call clears what it needs and overwrites the rest.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
int dls_compress_noalloc(const dls_params* p, const void* d_in, void* d_out, size_t out_cap,
                         size_t* out_bytes, dls_stream_t stream);

/* Decompress a device stream into a device field (Sec. 2.6, Algorithm 2).
 * d_out must hold nvars * nx*ny*nz*nt values of the stream's dtype; blocks
 * outside the stream's block range are left untouched.  Reads the header
 * with one synchronous copy and synchronizes `stream` at the end to report
 * DLS_ERR_CORRUPT. */
int dls_decompress(const void* d_comp, size_t comp_bytes, void* d_out, size_t out_cap,
                   dls_stream_t stream);

typedef struct {
  double max_abs_err;        /* max |orig - recon| over all points */
  int64_t n_over_bound;      /* points whose error exceeds their variable's pointwise bound */
  double nrmse;              /* 100 ||orig - recon||_2 / ||orig||_2 (Sec. 2.4), all variables */
  double ratio;              /* raw field bytes / stream bytes */
  double sum_sq_err, sum_sq; /* FP64 sums behind nrmse */
  int64_t n_points;
  int64_t n_blocks, n_raw_blocks, n_corr, n_esc;
  double mean_rank;          /* over non-raw blocks */
  int64_t bytes_header, bytes_basis, bytes_coeff, bytes_corr, bytes_esc, bytes_raw;
  double var_max_abs_err[8]; /* first 8 variables */
  double var_nrmse[8];
  int64_t var_over[8];
  double var_eb[8];          /* resolved bound per variable */
} dls_report;

/* Verify a reconstruction against the original (Sec. 2.4 metrics) and
 * describe the stream.  The bound per variable is read from the stream.
 * Returns DLS_ERR_BOUND_VIOLATED if a pointwise-mode stream has a point over
 * its bound; *h_out is filled in either case. */
int dls_verify(const void* d_orig, const void* d_recon, const void* d_comp, size_t comp_bytes,
               dls_report* h_out, dls_stream_t stream);

/* Stage entry points of the mixed-precision form, for exact tests of its
 * FP64-semantics decisions.  Device arrays of n elements.
 * dls_stage_quantize: q[i] = rint((double)c[i] / delta) (ties to even), the
 *   quantizer of Sec. 2.5's coefficients; ovf[i] = 1 where |c/delta| >= 2^24.
 * dls_stage_correct: the pointwise correction of a reconstruction xh against
 *   x with bound eb: k[i] = rint((x - xh) / 2eb) evaluated in FP64, or
 *   INT32_MIN where the point escapes (|x - xtilde| > eb or |k| > 2^20). */
int dls_stage_quantize(const float* d_c, int64_t n, double delta, int32_t* d_q, int32_t* d_ovf,
                       dls_stream_t stream);
int dls_stage_correct(const float* d_x, const float* d_xh, int64_t n, double eb, int32_t* d_k,
                      dls_stream_t stream);
/* The same correction through the code path a compression takes, so that
 * each path can be tested on identical inputs against the FP64 definition:
 *   DLS_CORR_PATH_EXACT:  the decision of the row-loading kernel (as
 *                         dls_stage_correct);
 *   DLS_CORR_PATH_SPARSE: the per-block kernel's sparse encode pass: elements
 *                         with |fl(x - xh)| below eb (1 - 1e-6), rounded down,
 *                         get k = 0 without a decision; the others take its
 *                         branch-free FP32 test and, where that test cannot
 *                         decide, the FP64 definition;
 *   DLS_CORR_PATH_DENSE:  the per-block kernel's dense encode pass: every
 *                         element takes the FP32 test, then the FP64
 *                         definition where the test cannot decide.
 * All three return exactly what dls_stage_correct returns. */
enum { DLS_CORR_PATH_EXACT = 0, DLS_CORR_PATH_SPARSE = 1, DLS_CORR_PATH_DENSE = 2 };
int dls_stage_correct_path(const float* d_x, const float* d_xh, int64_t n, double eb, int32_t path, int32_t* d_k,
                           dls_stream_t stream);

/* Block-rank MLP (not in the paper): 32 block features -> 64 -> 64 -> 1, ReLU,
 * BF16 weights with FP32 accumulation.  Parameters are DLS_MLP_NPARAM floats:
 * [mu 32][sigma 32][W1 64x32][b1 64][W2 64x64][b2 64][W3 64][b3 1], W row-major
 * (output x input); mu and sigma standardise the features (not trained).
 * Features of a block (computed in FP32/FP64 from its data and eigenvalues):
 *   0: log10(sum lambda / eps_l^2); 1..16: log10(sum_{i>=r} lambda_i / eps_l^2),
 *   r = 0..15; 17..24: sqrt(lambda_i / lambda_0), i = 1..8; 25: temporal and
 *   26: x gradient energy over ||X||^2; 27: log10(L delta^2 / 12 / eps_l^2);
 *   28: log10(value range / delta); 29: block size / 65536; 30: n / 16;
 *   31: the eigenvalue-tail rank estimate. */
#define DLS_MLP_NPARAM 6401
#define DLS_MLP_NFEAT 32

/* Loads the rank model on the current device (host array of DLS_MLP_NPARAM
 * floats; sigma entries must be > 0).  Weights are rounded to BF16. */
int dls_set_rank_model(const float* h_params, size_t count);

/* Features and exact ranks of every block (rank by the bisection of
 * Algorithm 1 in the FP32 mode; -1 for blocks stored raw).  d_feat: nb x 32
 * floats, d_rank: nb int32 (nb = blocks in the parameters' range).  Needs the
 * workspace dls_workspace_size(p) with p->precision = DLS_PREC_FP32. */
int dls_block_features(const dls_params* p, const void* d_in, float* d_feat, int32_t* d_rank, void* d_workspace,
                       size_t ws_bytes, dls_stream_t stream);

/* MLP on n feature rows (d_feat n x 32) -> d_y (n), weights rounded to BF16. */
int dls_mlp_forward(const float* d_params, const float* d_feat, int64_t n, float* d_y, dls_stream_t stream);

/* Gradient of the mean squared error over one minibatch (1 <= n <= 128):
 * d_grad (DLS_MLP_NPARAM floats, zero for mu and sigma), d_loss (1 float). */
int dls_mlp_grad(const float* d_params, const float* d_feat, const float* d_target, int64_t n, float* d_grad,
                 float* d_loss, dls_stream_t stream);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the MSE
 * of the predicted rank, minibatches of `batch` (<= 128) rows taken in the
 * order d_order[(s * batch + b) % n_order].  d_params and d_adam (2 x
 * DLS_MLP_NPARAM floats: first and second moments) are updated in place;
 * step0 is the number of steps already taken; d_loss (steps floats, may be
 * NULL) receives each step's minibatch loss.  Runs in one CTA. */
int dls_mlp_train(float* d_params, float* d_adam, const float* d_feat, const float* d_target, const int32_t* d_order,
                  int64_t n_order, int32_t steps, int32_t batch, float lr, int32_t step0, float* d_loss,
                  dls_stream_t stream);

/* Cycle counters of the last compression in this workspace by the
 * mixed-precision per-block kernel, summed over CTAs, in phase order: Gram
 * pass, FP32 Jacobi, FP64 refinement, Rayleigh-Ritz step, rank prediction,
 * encode pass at the predicted rank, exact pass tests, bisection fallback,
 * record packing; then three counts: blocks whose predicted rank was
 * accepted, blocks that fell back to the bisection, and FP64 re-evaluations
 * of E(r) taken because the FP32 estimate could not decide; then the cycles
 * spent waiting for staged tiles (included in the phases above; 0 for blocks
 * the row-loading kernel serves); then the number of blocks whose Gram ran on
 * the tensor cores (DLS_PREC_TF32X3).  count >= 14.  Synchronous copy. */
int dls_phase_cycles(const dls_params* p, const void* d_workspace, unsigned long long* h_cycles, int32_t count);

/* Stream header as a host struct (Sec. 2.7.2: the header and offset table
 * that make every record addressable).  Reads the header with one
 * synchronous copy from device memory; the eb, delta and step arrays hold the
 * resolved per-variable values (first nvars entries).  DLS_ERR_INVALID_ARG for
 * a null pointer or a stream shorter than the header or not 16-byte aligned,
 * DLS_ERR_CORRUPT when the header fails the decoder's checks (magic, version,
 * sizes, offsets), DLS_ERR_CUDA if the copy fails. */
typedef struct {
  int32_t version, nvars, dtype, eb_type, precision, rank_mode, rank_cap;
  int64_t dims[4];
  int32_t block[4];
  int64_t block_begin, block_end, total_blocks;
  uint64_t total_bytes;
  double eb[64], delta[64], step[64];
} dls_stream_info;
int dls_stream_info_get(const void* d_comp, size_t comp_bytes, dls_stream_info* h_info);

/* Fault injection for tests (no GPU fault is involved).  kind
 * DLS_FAULT_WITHHOLD_CHUNK: in every compression launched after this call
 * (plans: captured at dls_plan_create), the per-block kernel of the FP32 and
 * TF32X3 forms never issues the copy of the first staged chunk of block
 * `arg` (an index into the call's block range).  Its bounded wait for that
 * chunk runs out after about a second of SM clock, the kernel drains the
 * copies it did issue and ends, and the call returns DLS_ERR_TIMEOUT.
 * DLS_FAULT_NONE (arg ignored) switches the hook off.  Not thread-safe with
 * respect to concurrent compressions; meant for tests only. */
enum { DLS_FAULT_NONE = 0, DLS_FAULT_WITHHOLD_CHUNK = 1 };
int dls_set_fault_hook(int32_t kind, int64_t arg);

/* Static text for a DLS_* status ("unknown status" for other values). */
const char* dls_status_string(int status);

/* ------------------------------------------------------------------------
 * Global-basis mode: the method as Algorithm 1 states it (Sec. 2.3 Eq. 2-3,
 * Sec. 2.4 Eq. 4, Sec. 2.5 Eq. 5-6, Sec. 2.6), one basis per variable for
 * every patch of every snapshot, beside the block-local mode above.
 *   step 1: Q (S x M) holds S patches of the first snapshot (rows, x fastest
 *           within a patch) at the caller's origins; the modes Phi are the
 *           eigenvectors of Q^T Q by decreasing eigenvalue (the right singular
 *           vectors of Q), each signed so that its largest-magnitude
 *           component is positive (the lowest index on ties);
 *   step 2: eps = eps_t ||u|| / 100 over the variable (all snapshots),
 *           eps_l^2 = eps^2 M / K, delta = eps / sqrt(K);
 *   step 3: per patch of every snapshot (tiling from the origin): alpha =
 *           Phi^T u, q = rint(alpha / delta), the coefficients ranked by
 *           decreasing |alpha| (index order on ties), and the smallest kept
 *           count n by bisection over [0, M] with pass(n) := ||u - sum_{s<n}
 *           q_s delta phi_s||^2 <= eps_l^2 (the kept modes added in kept order).
 * Everything in FP64.  Patches are m x m x m (m x m when nz == 1), M <= 128;
 * the extents must be multiples of the patch.  One float32 variable per call,
 * laid out (nt, nz, ny, nx).
 * Stream ("DLSG", little-endian): header of 80 bytes (magic, u32 version 1,
 * M, px, py, pz, u64 nx, ny, nz, nt, f64 eps_l^2, f64 delta, u64 records),
 * the basis M x M float64 mode after mode, (records + 1) u64 offsets (an
 * exclusive scan of the record sizes), then the records in (t, z, y, x) patch
 * order: u32 n, u8 wv, three zero bytes, n mode indices of bit_width(M - 1)
 * bits then n zigzag(q) of wv bits, LSB first in 32-bit words, padded to 8
 * bytes. */
typedef struct {
  int64_t dims[4];      /* nx, ny, nz, nt */
  int32_t m;            /* patch edge */
  double eps_t;         /* NRMSE target in percent (> 0) */
  int64_t nsample;      /* S: rows of the sample matrix (>= 1) */
} dls_gb_params;

/* Worst-case stream bytes; 0 for invalid parameters. */
size_t dls_gb_bound(const dls_gb_params* p);
/* Device workspace bytes dls_gb_compress needs (256-byte aligned). */
size_t dls_gb_workspace_size(const dls_gb_params* p);
/* d_in: the variable (nt, nz, ny, nx) float32 on the device; d_origins: S x 3
 * int64 (x, y, z) patch origins in the first snapshot, each patch inside it
 * (else DLS_ERR_INVALID_ARG, checked on the device).  On success *out_bytes
 * is the stream size; DLS_ERR_CAPACITY sets it to the size needed.
 * Synchronizes `stream`. */
int dls_gb_compress(const dls_gb_params* p, const float* d_in, const int64_t* d_origins, void* d_out, size_t out_cap,
                    size_t* out_bytes, void* d_workspace, size_t ws_bytes, dls_stream_t stream);
/* The variable from a DLSG stream, in FP64 (each patch rebuilt as the sum of
 * its kept modes in kept order, Sec. 2.6): d_out holds nt*nz*ny*nx doubles.
 * DLS_ERR_CORRUPT for a stream that fails validation.  Synchronizes `stream`. */
int dls_gb_decompress(const void* d_comp, size_t comp_bytes, double* d_out, size_t out_count, dls_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
