// Internal definitions shared by the CUDA translation units of libdls.
// Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/dls.h"

namespace dls {

// ---------------------------------------------------------------- stream format
// Global header (128 bytes), per-variable table (32 bytes each), u64 offset
// table (nb + 1 entries, relative to the payload), then 16-byte aligned
// records.  Layout of a record: see the packer in k_pack.cu.
constexpr uint32_t kMagic = 0x31534C44u;  // "DLS1"
constexpr uint32_t kVersion = 1u;
constexpr int kHdr = 128;
constexpr int kVarRec = 32;
constexpr uint32_t kFlagRaw = 1u, kFlagSpatial = 2u, kFlagDense = 4u;
// Rice-coded correction section (the lossless stage, corr_codec = 1): see k_rice.cu.
constexpr uint32_t kFlagRice = 8u;
constexpr int kRiceChunk = 1024;           // elements per independently decodable chunk
constexpr int kRiceMaxKr = 20;             // Rice parameters tried: 0..20
// Block metadata only (never in a record): the record waits in its staging
// slot for the deferred packer, which writes it at its stream offset.
constexpr uint32_t kFlagDeferred = 1u << 8;
constexpr double kQmaxF32 = 16777216.0;    // |c/delta| must stay below 2^24 (f32 fields)
constexpr double kQmaxF64 = 1073741824.0;  // 2^30 (f64 fields)
constexpr double kKmax = 1048576.0;        // corrections beyond 2^20 steps become escapes
constexpr int32_t kEscape = INT32_MIN;     // escape marker in the correction workspace
constexpr int kMaxVars = 64;
constexpr int kMaxN = 32;                  // largest Gram order

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- plan
struct Plan {
  int32_t nvars, dtype, eb_type, rank_cap, precision, rank_mode;
  int64_t dims[4];
  int32_t block[4];
  int64_t nbk[4];          // blocks per axis
  int64_t nb_total;        // blocks in the field
  int64_t b0, nb;          // block range processed: [b0, b0 + nb)
  int64_t K;               // points per variable
  int64_t P;               // points per timestep (nx*ny*nz)
  int32_t nmax, lmax;      // largest Gram order / long side over blocks
  int64_t nmax_full;       // Gram order of a full block
  int64_t offsets_pos, payload_pos;   // byte positions in the stream
  int64_t pt_base, pt_count;          // point range of the processed blocks (workspace indexing)
  int32_t basis_n;                    // Gram order of the fixed basis (0: none)
  int32_t has_gstats;                 // bound statistics given by the caller (a part of a field)
  int32_t corr_codec;                 // 1: Rice-coded correction sections where smaller
  double kbound;                      // points per variable the bound refers to (K, or the whole field's)
  double eb_user[kMaxVars];
};

struct Geom {
  int32_t v, sx, sy, sz, st, n, side;
  int64_t x0, y0, z0, t0;
  int64_t M, T, N, L;
  int64_t pt_off;          // offset of the block's points in point-ordered workspaces
};

__host__ __device__ inline Geom block_geom(const Plan& p, int64_t b) {
  Geom g;
  int64_t ix = b % p.nbk[0]; b /= p.nbk[0];
  int64_t iy = b % p.nbk[1]; b /= p.nbk[1];
  int64_t iz = b % p.nbk[2]; b /= p.nbk[2];
  int64_t it = b % p.nbk[3]; b /= p.nbk[3];
  g.v = (int32_t)b;
  g.x0 = ix * p.block[0]; g.y0 = iy * p.block[1]; g.z0 = iz * p.block[2]; g.t0 = it * p.block[3];
  int64_t rx = p.dims[0] - g.x0, ry = p.dims[1] - g.y0, rz = p.dims[2] - g.z0, rt = p.dims[3] - g.t0;
  g.sx = (int32_t)(rx < p.block[0] ? rx : p.block[0]);
  g.sy = (int32_t)(ry < p.block[1] ? ry : p.block[1]);
  g.sz = (int32_t)(rz < p.block[2] ? rz : p.block[2]);
  g.st = (int32_t)(rt < p.block[3] ? rt : p.block[3]);
  g.M = (int64_t)g.sx * g.sy * g.sz;
  g.T = g.st;
  g.N = g.M * g.T;
  if (g.T <= g.M) { g.side = 0; g.n = (int32_t)g.T; g.L = g.M; }
  else { g.side = 1; g.n = (int32_t)g.M; g.L = g.T; }
  // Blocks are ordered (v, t, z, y, x); the points of all earlier blocks are
  // v*K + t0*P + st*(z0*nx*ny + sz*(y0*nx + sy*x0)).
  g.pt_off = (int64_t)g.v * p.K + g.t0 * p.P +
             (int64_t)g.st * (g.z0 * p.dims[0] * p.dims[1] + (int64_t)g.sz * (g.y0 * p.dims[0] + (int64_t)g.sy * g.x0));
  return g;
}

// Global index of block element (spatial ls, time lt).
__host__ __device__ inline int64_t elem_index(const Plan& p, const Geom& g, int64_t ls, int64_t lt) {
  int64_t lx = ls % g.sx, r = ls / g.sx;
  int64_t ly = r % g.sy, lz = r / g.sy;
  return (int64_t)g.v * p.K + (g.t0 + lt) * p.P + (g.z0 + lz) * p.dims[0] * p.dims[1] +
         (g.y0 + ly) * p.dims[0] + (g.x0 + lx);
}

// Global index of block-matrix entry A[l][j].
__host__ __device__ inline int64_t a_index(const Plan& p, const Geom& g, int64_t l, int j) {
  return g.side == 0 ? elem_index(p, g, l, j) : elem_index(p, g, j, l);
}
// Element order inside a block: e = t_local * M + s_local.
__host__ __device__ inline int64_t a_elem(const Geom& g, int64_t l, int j) {
  return g.side == 0 ? (int64_t)j * g.M + l : l * g.M + j;
}

// ---------------------------------------------------------------- per-variable state (device)
struct VarInfo {
  double eb_user, eb, delta, step;  // resolved bound, quantization step, correction step
  double sumsq;                     // sum of squares (NRMSE mode)
  unsigned long long minkey, maxkey;// ordered keys for min / max (REL_RANGE mode)
};

// ---------------------------------------------------------------- per-block result
struct BlockMeta {
  int32_t r, flags, wk, ib;
  int32_t ncorr, nesc;
  int32_t nprobes, rcap;
  int64_t nbytes;
  uint8_t wq[kMaxN];
};

// Status words written by kernels and read by the host after one sync.
struct Status {
  unsigned int nonfinite;
  unsigned int capacity;
  unsigned int corrupt;
  unsigned int timeout;
  unsigned long long total_bytes;
  unsigned long long pad[5];
};

// ---------------------------------------------------------------- workspace
struct Work {
  BlockMeta* meta;      // nb
  double* vst;          // nb * nmax * nmax (stored basis, dtype-rounded, n x rcap row-major)
  int32_t* q;           // point-ordered: block b at pt_off, L x rcap column-major (k*L + l)
  int32_t* kc;          // point-ordered: block b at pt_off, element order e
  unsigned long long* offsets;  // nb + 1
  VarInfo* vars;        // nvars
  Status* status;
  const double* basis;  // basis_n x basis_n fixed modes (null: none)
  const double* gstats; // nvars x 4 statistics of the whole field (null: from the field passed)
};

// Per block, the Rice stage's choice: on, parameter kr, value width wv and
// the coded words (the section is 2 + chunks + words words).
struct RiceInfo {
  uint32_t words;
  int32_t kr, wv, on;
};
// Per chunk of a record's corrections: c[i] = runs of zeros with bit i set,
// and the nonzeros, so that the chunk's code length is known for every kr.
struct RiceChunk {
  uint16_t c[11];
  uint16_t nnz;
  uint32_t first;   // entry-list sources: the chunk's first entry
};
__host__ __device__ inline int64_t rice_chunks_per_block(const Plan& p) {
  return cdiv((int64_t)p.block[0] * p.block[1] * p.block[2] * p.block[3], kRiceChunk);
}

// ordered key for doubles (monotone map to unsigned)
__host__ __device__ inline unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
__host__ __device__ inline double bitsd(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
__host__ __device__ inline unsigned long long dkey(double x) {
  unsigned long long u = dbits(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double dunkey(unsigned long long k) {
  return bitsd((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k);
}

__device__ __forceinline__ uint32_t zigzag(int32_t v) { return ((uint32_t)v << 1) ^ (uint32_t)(v >> 31); }
__device__ __forceinline__ int32_t unzigzag(uint32_t z) { return (int32_t)((z >> 1) ^ (0u - (z & 1u))); }
__host__ __device__ inline int bit_width(uint32_t v) {
#ifdef __CUDA_ARCH__
  return 32 - __clz(v);
#else
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
#endif
}

// Record layout arithmetic shared by the size computation and the packer.
struct RecLayout {
  int64_t off_wq, off_v, off_q, off_c, off_ei, off_ev, size;
  int64_t corr_words;
  int dense;
};
__host__ __device__ inline RecLayout rec_layout(int r, int n, int64_t L, int64_t N, int es,
                                                const uint8_t* wq, int wk, int ib, int64_t ncorr,
                                                int64_t nesc) {
  RecLayout o;
  o.off_wq = 16;
  o.off_v = o.off_wq + align_up(r, 8);
  o.off_q = o.off_v + align_up((int64_t)n * r * es, 8);
  int64_t qwords = 0;
  for (int c = 0; c < r; ++c) qwords += (L * wq[c] + 31) / 32;
  int64_t dense_w = (N * wk + 31) / 32, sparse_w = (ncorr * (ib + wk) + 31) / 32;
  o.dense = (wk > 0) && (dense_w < sparse_w);
  o.corr_words = wk == 0 ? 0 : (o.dense ? dense_w : sparse_w);
  o.off_c = o.off_q + align_up(qwords * 4, 8);
  o.off_ei = o.off_c + align_up(o.corr_words * 4, 8);
  o.off_ev = o.off_ei + align_up(nesc * 4, 8);
  o.size = align_up(o.off_ev + align_up(nesc * es, 8), 16);
  return o;
}
__host__ __device__ inline int64_t raw_record_bytes(int64_t N, int es) { return align_up(16 + N * es, 16); }
// The layout of the same record with a Rice-coded correction section of
// `rice_words` coded words: [count, kr | wv << 8, chunk bit offsets, words].
__host__ __device__ inline RecLayout rice_layout(RecLayout o, int64_t N, int64_t rice_words, int64_t nesc, int es) {
  o.dense = 0;
  o.corr_words = 2 + cdiv(N, kRiceChunk) + rice_words;
  o.off_ei = o.off_c + align_up(o.corr_words * 4, 8);
  o.off_ev = o.off_ei + align_up(nesc * 4, 8);
  o.size = align_up(o.off_ev + align_up(nesc * es, 8), 16);
  return o;
}

// Workspace of the mixed-precision form.
struct MixedWork {
  BlockMeta* meta;
  unsigned long long* offsets;
  VarInfo* vars;
  Status* status;
  uint8_t* staging;     // per-block record slots: align16(pt_rel * 4) + 48 * bi
  int32_t* q_scr;       // ctas x kMaxMixedN x lmax
  int8_t* k8_scr;       // ctas x nptmax
  int32_t* k32_scr;     // ctas x nptmax
  uint32_t* bit_scr;    // ctas x nptmax / 32: nonzero-correction bitmap (full blocks)
  float* feat;          // nb x 32
  int32_t* ranks;       // nb
  int64_t lmax, nptmax;
  int ctas;
  unsigned long long* phase;   // ctas x kMixedPhases cycle counters
  uint8_t* fast;        // per-block state of the tile route's phase kernels (tile_fast_bytes)
  // The field with its x lines padded to `pitch` floats (a multiple of 4), for
  // fields whose x extent is not: the staged kernels' tensor map reads this
  // copy, so every chunk comes in by TMA (null and 0 when not used).
  float* pitched;
  int64_t pitch;
};
// Padded x-line length of the pitched copy for a plan, or 0 when the plan
// reads its field directly: a float32 field through the staged kernels, over
// its whole block range, whose x extent is not a multiple of 4 while the block
// width is (a TMA box row must be a multiple of 16 bytes).
int64_t pitched_row(const Plan& P, bool staged);
constexpr int kMaxMixedN = 16;
constexpr int kMixedPhases = 14;

// Block-rank MLP: 32 features -> 64 -> 64 -> 1 (ReLU).  Parameter vector layout
// (floats): [mu 32][sigma 32][W1 64x32][b1 64][W2 64x64][b2 64][W3 64][b3 1].
constexpr int kMlpF = 32, kMlpH = 64;
constexpr int kMlpOffMu = 0, kMlpOffSig = kMlpF, kMlpOffW1 = 2 * kMlpF;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpH * kMlpF;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpH;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpH * kMlpH;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpH;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpH;
constexpr int kMlpNParam = kMlpOffB3 + 1;   // 6401
// rank modes of the kernel
constexpr int kRankSearch = 0, kRankMlp = 1, kRankTail = 2;

// Validates the parameters and builds the plan (dls_api.cu); DLS_OK or the
// status dls_compress would return for them.
int make_plan(const dls_params* p, Plan* out);

// Test hook (dls_set_fault_hook): the block, in a call's block range, whose
// first staged chunk the per-block kernel never copies; -1 for none.
int64_t fault_withheld_block();

// ---------------------------------------------------------------- launchers (defined in .cu files)
int launch_mixed_compress(const Plan& p, const void* d_in, const MixedWork& w, int learned, int variant,
                          int spatial_only, cudaStream_t s);
// Occupancy forms of the per-block kernels, one per shape class of a
// compression's blocks (1: the form built for 2 CTAs per SM, with more
// registers per thread; 2: the form built for 4).  `whole`: the blocks of the
// full block shape that k_enc encodes at the predicted rank.  `rest`: what
// k_tile and k_mixed take -- edge blocks of smaller shapes, predictions k_enc
// rejects, blocks whose Gram side is space, every block in the search mode;
// 0 there means the 2-CTA form behind k_enc (a short list) and the 4-CTA form
// when k_tile takes every block.  Both forms run the same code, so the choice
// changes the time and never a byte of the stream.
struct Occupancy {
  int whole;
  int rest;
};
constexpr Occupancy kOccDefault{2, 0};

// Records ev on s: as an event node of the graph while s is being captured
// (its time is then read after each replay), as a plain record otherwise (the
// external form is refused outside a capture).
inline cudaError_t record_marker(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// pev (optional): four events recorded after k_gram, k_eig, the
// Rayleigh-Ritz kernels and k_enc (for the phase timing of captured plans).
int launch_tile_compress(const Plan& p, const void* d_in, const MixedWork& w, int learned, Occupancy occ,
                         cudaStream_t s, int64_t blo = 0, int64_t bhi = -1, const cudaEvent_t* pev = nullptr);
bool tile_chunk_box(const Plan& p, int* bxb, int* yc, int* zc, int* bt);
size_t tile_fast_bytes(int64_t nb);
int launch_compact(const Plan& p, const MixedWork& w, void* d_out, cudaStream_t s);
int launch_pack_tile(const Plan& p, const MixedWork& w, const void* d_in, void* d_out, cudaStream_t s);
size_t mixed_smem_bytes();
int launch_mlp_train(float* params, float* adam, const float* feat, const float* target, const int32_t* order,
                     int64_t n_order, int steps, int B, float lr, int step0, float* loss, cudaStream_t s);
int launch_mlp_grad(const float* params, const float* feat, const float* target, int B, float* grad, float* loss,
                    cudaStream_t s);
int launch_mlp_forward(const float* params, const float* feat, int64_t n, float* y, cudaStream_t s);
int mlp_max_batch();
bool rank_model_loaded();
int launch_stage_quantize(const float* c, int64_t n, double delta, int32_t* q, int32_t* ovf, cudaStream_t s);
int launch_stage_correct(const float* x, const float* xh, int64_t n, double eb, int path, int32_t* k,
                         cudaStream_t s);
int launch_plain_compress(const Plan& p, const void* d_in, const Work& w, cudaStream_t s);
int launch_scan(const Plan& p, const Work& w, size_t out_cap, void* d_out, cudaStream_t s);
int launch_pack(const Plan& p, const void* d_in, const Work& w, void* d_out, size_t out_cap, cudaStream_t s);
int launch_rice(const Plan& p, const Work& w, const uint8_t* s0, RiceInfo* info, RiceChunk* chunks, size_t out_cap,
                void* d_out, cudaStream_t s);
int launch_stats_resolve(const Plan& p, const void* d_in, const Work& w, double* partial, cudaStream_t s);
int launch_field_stats(const Plan& p, const void* d_in, const Work& w, double* partial, double* h_stats,
                       cudaStream_t s);
int stats_partial_doubles(const Plan& p);
int launch_decode(const Plan& p, const void* d_comp, unsigned long long comp_bytes, void* d_out, Status* st,
                  cudaStream_t s);
int launch_verify(const Plan& p, const void* d_orig, const void* d_recon, const void* d_comp,
                  unsigned long long comp_bytes, double* acc, cudaStream_t s);

}  // namespace dls
