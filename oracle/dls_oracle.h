/*
 * dls_oracle.h -- plain FP64 CPU oracle for Discontinuous DLS block compression.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) includes, links or calls this code.  Only the tests,
 * __graft_entry__.smoke() and the CPU-baseline leg of bench.py use it.
 * It shares no header, helper, table or constant generator with the CUDA path.
 *
 * What it computes (paper: "A Data-Informed Local Subspaces Method for
 * Error-Bounded Lossy Compression", arXiv 2601.20113):
 *   - blocks (patches) tile the space-time field, Sec. 2.2 / Algorithm 1 step 2;
 *   - each block's basis is the set of right singular vectors of its data
 *     matrix, obtained the cross-product way (Gram matrix + symmetric
 *     eigensolve), Sec. 2.3 Eq. (2)-(3) and Sec. 2.7.1;
 *   - coefficients are the projection S = C^T P, Sec. 2.5 Eq. (5);
 *   - the retained set is the smallest significance-ordered prefix meeting the
 *     local L2 tolerance, found by bisection, Sec. 2.5 Eq. (6), Algorithm 1;
 *   - the local tolerance follows Sec. 2.4 Eq. (4);
 *   - reconstruction and assembly follow Sec. 2.6 and Algorithm 2;
 *   - the stream (addressable header, offset table from an exclusive scan,
 *     tightly packed per-block arrays) follows Sec. 2.7.2.
 * Quantization of coefficients (in place of bit-grooming) and the pointwise
 * correction pass are readings of the paper's L-infinity metric (Sec. 2.4)
 * and of its bit-grooming step (Sec. 2.5), stated where they are defined.
 *
 * All functions are plain C, single-threaded per block; or_compress and
 * or_decompress run blocks in parallel with OpenMP.
 */
#ifndef DLS_ORACLE_H
#define DLS_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_F32 = 0, OR_F64 = 1 };
enum { OR_EB_ABS = 0, OR_EB_REL_RANGE = 1, OR_EB_NRMSE = 2 };
enum {
  OR_OK = 0, OR_ERR_INVALID_ARG = -1, OR_ERR_CAPACITY = -2, OR_ERR_NONFINITE = -3,
  OR_ERR_CORRUPT = -4
};

typedef struct {
  int32_t nvars;
  int64_t dims[4];      /* nx, ny, nz, nt (x fastest) */
  int32_t block[4];     /* bx, by, bz, bt */
  int32_t dtype;        /* OR_F32 / OR_F64 */
  int32_t eb_type;      /* OR_EB_* */
  const double* eb;     /* nvars user values */
  int32_t rank_cap;
  int64_t block_begin, block_end;   /* [begin,end); end < 0 means all */
  /* Fixed basis (Sec. 4, the SVD / cosine / random comparison): when basis is
     not null, blocks whose Gram order equals basis_n use its columns
     (basis[a * basis_n + k] = component a of mode k, orthonormal) in the given
     order instead of their own eigenvectors; other blocks are unchanged. */
  const double* basis;
  int32_t basis_n;
  /* 0: corrections as dense or index list (the stream the CUDA library
     writes); 1: a Rice-coded section too, wherever it is smaller (a proposed
     format, see or_pack_record). */
  int32_t corr_codec;
  /* Statistics of the whole field when `field` is one part of it (a z-slab
     of a data-distributed field, Sec. 2.7.1): nvars x 4 doubles, per variable
     {min, max, sum of squares, number of points}.  Bound resolution takes the
     range, the norm and K from here instead of from the part, so the part's
     records are those of the whole field.  Null: the field is whole. */
  const double* global_stats;
} or_params;

/* Geometry of one block. */
typedef struct {
  int32_t v;
  int64_t x0, y0, z0, t0;
  int32_t sx, sy, sz, st;
  int64_t M, T, N;        /* spatial points, timesteps, N = M*T */
  int64_t L;              /* long side */
  int32_t n;              /* short side (Gram order) */
  int32_t side;           /* 0 = temporal basis (T <= M), 1 = spatial basis */
} or_geom;

/* Per-variable bound resolution (Sec. 2.4). */
typedef struct {
  double eb_user;   /* as given */
  double eb;        /* pointwise bound (ABS/REL) or global L2 budget eps (NRMSE) */
  double delta;     /* coefficient quantization step */
  double step;      /* correction step 2*eb (0 in NRMSE mode) */
  double norm2;     /* sum of squares of the variable (NRMSE mode only) */
  int64_t K;        /* points of the variable */
} or_var;

/* Per-block trace for tests. */
typedef struct {
  int32_t n, side, rcap, r, raw, sweeps, nprobes, lin_r, overflow;
  int32_t wk, ib, dense;
  int64_t L, N, n_corr, n_esc, nbytes;
  double el2;
  double E[33];          /* E(r) for probed r, NaN otherwise */
  int32_t probe_r[8];
} or_trace;

int64_t or_num_blocks(const or_params* p);
int     or_block_geom(const or_params* p, int64_t b, or_geom* g);
int     or_validate(const or_params* p);
int     or_resolve(const or_params* p, const void* field, or_var* vars);

/* Stage functions on one block matrix A (L x n, row-major doubles). */
void    or_gather(const or_params* p, const void* field, const or_geom* g, double* A);
void    or_gram(const double* A, int64_t L, int n, double* G);
int     or_jacobi(const double* G, int n, double* lam, double* V);   /* returns sweeps */
void    or_round_basis(const double* V, int n, int r, int dtype, double* Vst);
void    or_project(const double* A, int64_t L, int n, const double* Vst, int r, double* C);
int     or_quantize(const double* C, int64_t cnt, double delta, int dtype, int32_t* q);
void    or_decode(const int32_t* q, int64_t L, int rq, int r, const double* Vst, int n,
                  int dtype, double delta, double* D);
double  or_block_err(const double* A, const double* D, int64_t L, int n);
void    or_correct(const double* A, const double* D, int64_t L, int n, int side, int64_t M,
                   int dtype, double eb, double step, int32_t* k, uint8_t* esc);

/* One block end to end; writes its record into rec (capacity rec_cap) and
 * returns the record size in bytes (or a negative status).  Optional
 * intermediate outputs may be NULL. */
int64_t or_block_compress(const or_params* p, const void* field, int64_t b, const or_var* vars,
                          uint8_t* rec, int64_t rec_cap, or_trace* tr,
                          double* G_out, double* lam_out, double* V_out, double* Vst_out,
                          int32_t* q_out, int32_t* k_out, int want_linear);

int64_t or_max_record_bytes(const or_params* p, int64_t b);
int64_t or_compress_bound(const or_params* p);
int     or_compress(const or_params* p, const void* field, void* out, int64_t cap,
                    int64_t* out_bytes, or_trace* traces, int nthreads);
int     or_decompress(const void* stream, int64_t bytes, void* out, int64_t out_cap, int nthreads);

/* Standalone record packer, for bit-exact packer tests on identical inputs.
 * q is L x r (row-major, leading dimension r), k has N entries in element
 * order, esc marks escaped points (raw values taken from A). */
int64_t or_pack_record(int r, int side, int n, int64_t L, int64_t M, int dtype,
                       const double* Vst, const int32_t* q, const int32_t* k,
                       const uint8_t* esc, const double* A, uint8_t* rec, int64_t cap, int corr_codec);

/* Rice-coded corrections, the record section or_pack_record takes with
 * corr_codec = 1 (the layout is described in dls_oracle.c): exact size in bits, the
 * parameters with the fewest bits, encoder (bits written, -1 if cap_words is
 * too small; off gets each chunk's bit offset) and decoder (0, or -1 for a
 * malformed section). */
int64_t or_rice_bits(const int32_t* k, int64_t N, int chunk, int kr, int wv);
void    or_rice_choose(const int32_t* k, int64_t N, int chunk, int* kr, int* wv);
int64_t or_rice_encode(const int32_t* k, int64_t N, int chunk, int kr, int wv, uint32_t* words,
                       int64_t cap_words, uint32_t* off);
int     or_rice_decode(const uint32_t* words, int64_t nwords, const uint32_t* off, int64_t N, int chunk,
                       int kr, int wv, int32_t* k);

/* Inverse of or_pack_record for one record of the given geometry (raw
 * records return their values in escval); 0 or OR_ERR_CORRUPT. */
int     or_parse_record(const uint8_t* rec, int64_t nbytes, int side, int n, int64_t L, int64_t M, int dtype,
                        int* r, int* flags, double* Vst, int32_t* q, int32_t* k, uint8_t* esc, double* escval);
/* Coefficients of the FP32 (mixed-precision) form: the shifted binary32
 * projection in its fixed order (see dls_oracle.c). */
void    or_project_f32(const double* A, int64_t L, int n, const double* Vst, int r, double* C);

#ifdef __cplusplus
}
#endif
#endif
