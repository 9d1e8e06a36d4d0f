// Mixed-precision compression path for float32 fields (Gram order n <= 16).
//
// One persistent kernel; each CTA takes blocks from an atomic counter and runs
// the whole per-block pipeline (Algorithm 1 step 3 of arXiv 2601.20113 in the
// pointwise-bound reading):
//   pass 1 (HBM): FP32 Gram G = A^T A (Sec. 2.7.1), block statistics
//   eigensolve: FP32 Jacobi, then one FP64 refinement step of the eigenpairs
//               (Ogita & Aishima, Japan J. Indust. Appl. Math. 35, 2018), so the
//               basis is the FP64-accurate eigenbasis of the FP32 Gram
//   rank: a predicted rank r^ is checked exactly (pass(r^) and not pass(r^-1));
//         otherwise the bisection of Algorithm 1 runs on E(r) for all r
//   pass 2 (L2): projection C = A Vst in FP32, quantization, decode, the two
//               checks and the pointwise correction
//   pack: the record is written into a per-block staging slot.
// Every stored decision (q, pass(r), k, escapes) has FP64 semantics: an FP32
// evaluation decides when its rounding error bound leaves no doubt, and the
// FP64 definition is evaluated otherwise, so the decisions equal the ones the
// FP64 definitions give on the same coefficients and reconstructions.
#include <mutex>

#include "mixed_common.cuh"

namespace dls {
namespace {

constexpr int kMT = 256;                 // threads per CTA
constexpr int kNP = NM * (NM + 1) / 2;   // packed upper triangle (136)
constexpr int kHalf = kNP / 2;           // pairs per thread group (68)
constexpr int kGrp = kMT / 2;            // threads per group
constexpr int kTab = 8192;               // row-offset table entries (spatial points of a block)

struct MxArgs {
  Plan P;
  const float* in;
  uint8_t* staging;        // per-block record slots
  BlockMeta* meta;
  VarInfo* vars;
  Status* status;
  int32_t* q_scr;          // per CTA: NM * lmax int32
  int8_t* k8_scr;          // per CTA: nmax_pts int8
  int32_t* k32_scr;        // per CTA: nmax_pts int32 (only for |k| > 127 or escapes)
  float* feat;             // nb x 32 block features (may be null)
  int32_t* ranks;          // nb: chosen rank (for analysis)
  int64_t lmax, nptmax;
  int learned;             // 1: check the predicted rank first
  unsigned long long* phase;   // per CTA: kPhases cycle counters (may be null)
  int spatial_only;            // 1: take only blocks whose Gram side is space
};
// Phases timed by the per-CTA cycle counters.
enum { kPhGram = 0, kPhJacobi, kPhRefine, kPhRR, kPhPredict, kPhEncode, kPhDecide, kPhSearch, kPhPack,
       kCntAccepted, kCntSearched, kCntExact, kPhTileWait, kCntTcGram, kPhases };

struct MxSmem {
  float G32[NM * NM];
  float Vj[NM * NM];
  double G64[NM * NM], X64[NM * NM], R64[NM * NM];
  double lam_t[NM];        // refined eigenvalues (unsorted)
  double lam[NM];          // sorted
  float Vst[NM * NM];      // stored basis, Vst[j*NM + k]
  float vsum[NM];          // sum_j Vst[j][k] (for the shifted projection)
  float red[8][kNP + 8];
  float ered[8][NM + 2];
  double Ered[NM + 2];
  int sh_warp[32];
  float st_min[8], st_max[8], st_gt[8], st_gx[8], st_rowmax[8];
  double st_sum[8];
  int wq[NM];
  int kmax, ncorr, nesc, ovf, nonfinite, bad;
  int64_t bi;
  int r_pred, r_fin, accepted;
  float featv[kMlpF];
  float mh1[kMlpH];
  unsigned nexact;
  // spatial offsets of the block's points relative to its origin, rebuilt when
  // the block shape changes (avoids 64-bit divisions on every row)
  int32_t rowoff[kTab];
  int tab_sx, tab_sy, tab_sz, tab_ok;
  int64_t base0;
  JacPairs jp;
};

// ---------------------------------------------------------------- rank model
// The trained block-rank MLP, one copy per device (set by dls_set_rank_model).
static __device__ MlpModel g_rank_model;

// ---------------------------------------------------------------- block geometry helpers
// Offset of spatial point ls from the block origin.
__device__ __forceinline__ int64_t spatial_off(const Plan& P, const Geom& g, int64_t ls) {
  const int64_t lx = ls % g.sx, r = ls / g.sx;
  const int64_t ly = r % g.sy, lz = r / g.sy;
  return lz * P.dims[0] * P.dims[1] + ly * P.dims[0] + lx;
}

// Builds S.rowoff for the block's shape if needed (all threads call).
__device__ void prepare_block(const MxArgs& a, MxSmem& S, const Geom& g) {
  const Plan& P = a.P;
  const bool same = S.tab_sx == g.sx && S.tab_sy == g.sy && S.tab_sz == g.sz;
  const bool fits = g.M <= kTab && (int64_t)g.sz * P.dims[0] * P.dims[1] < (1ll << 31);
  if (!same && fits) {
    for (int64_t ls = threadIdx.x; ls < g.M; ls += kMT) S.rowoff[ls] = (int32_t)spatial_off(P, g, ls);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S.tab_ok = fits ? 1 : 0;
    if (fits) { S.tab_sx = g.sx; S.tab_sy = g.sy; S.tab_sz = g.sz; }
    else { S.tab_sx = -1; }
    S.base0 = (int64_t)g.v * P.K + g.t0 * P.P + g.z0 * P.dims[0] * P.dims[1] + g.y0 * P.dims[0] + g.x0;
  }
  __syncthreads();
}

__device__ __forceinline__ int64_t soff(const MxArgs& a, const MxSmem& S, const Geom& g, int64_t ls) {
  return S.tab_ok ? (int64_t)S.rowoff[ls] : spatial_off(a.P, g, ls);
}

// Global index of block element (spatial ls, time lt).
__device__ __forceinline__ int64_t gidx(const MxArgs& a, const MxSmem& S, const Geom& g, int64_t ls, int64_t lt) {
  return S.base0 + lt * a.P.P + soff(a, S, g, ls);
}

__device__ __forceinline__ void load_row(const MxArgs& a, const MxSmem& S, const Geom& g, int64_t l, float* x) {
  if (g.side == 0) {
    const float* p = a.in + S.base0 + soff(a, S, g, l);
#pragma unroll
    for (int j = 0; j < NM; ++j) x[j] = (j < g.n) ? __ldg(p + (int64_t)j * a.P.P) : 0.0f;
  } else {
    const float* p = a.in + S.base0 + l * a.P.P;
#pragma unroll
    for (int j = 0; j < NM; ++j) x[j] = (j < g.n) ? __ldg(p + soff(a, S, g, j)) : 0.0f;
  }
}

// Fixed-order CTA reduction of `cnt` per-thread floats (cnt <= NM + 2); results in S.Ered (double).
__device__ void cta_reduce_floats(MxSmem& S, float* v, int cnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = 0; i < NM + 2; ++i) {
    if (i >= cnt) break;
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) S.ered[warp][i] = x;
  }
  __syncthreads();
  if (tid < cnt) {
    float s = 0.0f;
    for (int w = 0; w < kMT / 32; ++w) s = __fadd_rn(s, S.ered[w][tid]);
    S.Ered[tid] = (double)s;
  }
  __syncthreads();
}

// First-order orthonormalisation in FP64 (all threads): X <- X (I + R/2),
// R = I - X^T X.  The FP32 Jacobi's eigenvectors are orthonormal to about
// 1e-5; this step takes that to its square, below the rounding of the stored
// modes to binary32.
__device__ void reorth64(MxSmem& S, int n) {
  const int tid = threadIdx.x;
  const int i = tid / NM, j = tid % NM;
  const bool act = i < n && j < n;
  if (act) {
    double rr = 0.0;
    for (int k = 0; k < n; ++k) rr = fma(S.X64[k * NM + i], S.X64[k * NM + j], rr);
    S.R64[i * NM + j] = (i == j ? 1.0 : 0.0) - rr;
  }
  __syncthreads();
  double xn = 0.0;
  if (act) {
    xn = S.X64[i * NM + j];
    for (int k = 0; k < n; ++k) xn = fma(S.X64[i * NM + k], 0.5 * S.R64[k * NM + j], xn);
  }
  __syncthreads();
  if (act) S.X64[i * NM + j] = xn;
  __syncthreads();
}

// Sort (stable, descending, lambda < 0 -> 0), sign-normalise, round to f32 (warp 0).
__device__ void order_basis(MxSmem& S, int n, int lane) {
  if (lane < n) {
    const int k = lane;
    double dk = S.lam_t[k];
    dk = dk < 0.0 ? 0.0 : dk;
    int pos = 0;
    for (int j = 0; j < n; ++j) {
      double dj = S.lam_t[j];
      dj = dj < 0.0 ? 0.0 : dj;
      if (dj > dk || (dj == dk && j < k)) ++pos;
    }
    int imax = 0;
    double amax = -1.0;
    for (int a = 0; a < n; ++a) {
      const double av = fabs(S.X64[a * NM + k]);
      if (av > amax) { amax = av; imax = a; }
    }
    const bool neg = S.X64[imax * NM + k] < 0.0;
    S.lam[pos] = dk;
    double cs = 0.0;
    for (int a = 0; a < n; ++a) {
      const double v = S.X64[a * NM + k];
      const float vf = __double2float_rn(neg ? -v : v);
      S.Vst[a * NM + pos] = vf;
      cs += (double)vf;
    }
    S.vsum[pos] = (float)cs;
  }
  __syncwarp();
}

// ---------------------------------------------------------------- passes
// Projection + quantization of one row for columns k < kq; fills chat.
__device__ __forceinline__ void row_coeffs(const MxSmem& S, const float* x, int n, int kq, double delta,
                                           float inv_delta, float delta_f, int32_t* q, float* chat, int& ovf) {
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    q[k] = 0;
    chat[k] = 0.0f;
    if (k < kq) {
      // shifted by the row's first value: the differences are exact when the
      // row carries a large common part, so no cancellation error remains.
      // Four partial sums over j mod 4, combined as (s0 + s1) + (s2 + s3):
      // the coefficient definition the staged-tile kernel uses as well.
      const float a0 = x[0];
      float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int j = 0; j < NM; ++j)
        if (j < n) s4[j & 3] = __fmaf_rn(__fsub_rn(x[j], a0), S.Vst[j * NM + k], s4[j & 3]);
      const float c = __fmaf_rn(a0, S.vsum[k], __fadd_rn(__fadd_rn(s4[0], s4[1]), __fadd_rn(s4[2], s4[3])));
      q[k] = quant_exact(c, delta, inv_delta, ovf);
      chat[k] = __fmul_rn(__int2float_rn(q[k]), delta_f);
    }
  }
}

// pass computing E(r) for every r in [0, rcap] (FP32 estimates into S.Ered)
__device__ void pass_all_errors(const MxArgs& a, MxSmem& S, const Geom& g, int rcap, double delta, float inv_delta,
                                float delta_f, int& ovf) {
  const int tid = threadIdx.x, n = g.n;
  float E[NM + 1];
#pragma unroll
  for (int r = 0; r <= NM; ++r) E[r] = 0.0f;
  for (int64_t l = tid; l < g.L; l += kMT) {
    float x[NM];
    load_row(a, S, g, l, x);
    int32_t q[NM];
    float ch[NM];
    row_coeffs(S, x, n, rcap, delta, inv_delta, delta_f, q, ch, ovf);
    float acc[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) { acc[j] = 0.0f; if (j < n) E[0] = __fmaf_rn(x[j], x[j], E[0]); }
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      if (k < rcap) {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            acc[j] = __fmaf_rn(ch[k], S.Vst[j * NM + k], acc[j]);
            const float d = __fsub_rn(x[j], acc[j]);
            E[k + 1] = __fmaf_rn(d, d, E[k + 1]);
          }
        }
      }
    }
  }
  cta_reduce_floats(S, E, rcap + 1);
}

// FP64 evaluation of E(r) in the fixed order of the definition (per column,
// rows in chunks of 32, chunk sums in order, column sums in order).  Used only
// when the FP32 estimate cannot decide.  Uses S.red as scratch (kMT doubles).
__device__ double exact_error(const MxArgs& a, MxSmem& S, const Geom& g, int r, double delta, float inv_delta,
                              float delta_f) {
  const int tid = threadIdx.x, n = g.n;
  const int64_t nch = cdiv(g.L, 32);
  double* part = reinterpret_cast<double*>(&S.red[0][0]);   // 8*(kNP+8)*4 B >= kMT * 8 B
  double colsum = 0.0;   // held by thread j < n
  for (int j = 0; j < n; ++j) {
    for (int64_t c0 = 0; c0 < nch; c0 += kMT) {
      const int64_t c = c0 + tid;
      if (c < nch) {
        double pc = 0.0;
        const int64_t l1 = (c + 1) * 32 < g.L ? (c + 1) * 32 : g.L;
        for (int64_t l = c * 32; l < l1; ++l) {
          float x[NM];
          load_row(a, S, g, l, x);
          int32_t q[NM];
          float ch[NM];
          int ovf = 0;
          row_coeffs(S, x, n, r, delta, inv_delta, delta_f, q, ch, ovf);
          float acc = 0.0f;
          for (int k = 0; k < r; ++k) acc = __fmaf_rn(ch[k], S.Vst[j * NM + k], acc);
          const double d = __dsub_rn((double)x[j], (double)acc);
          pc = __fma_rn(d, d, pc);
        }
        part[tid] = pc;
      }
      __syncthreads();
      if (tid == j) {
        const int64_t cend = (nch - c0) < kMT ? (nch - c0) : kMT;
        for (int64_t cc = 0; cc < cend; ++cc) colsum = __dadd_rn(colsum, part[cc]);
      }
      __syncthreads();
    }
  }
  // column sums in order: thread j holds column j
  __shared__ double cs[NM];
  if (tid < n) cs[tid] = colsum;
  __syncthreads();
  double E = 0.0;
  for (int j = 0; j < n; ++j) E = __dadd_rn(E, cs[j]);
  __syncthreads();
  return E;
}

// pass(r): E(r) <= el2 with FP64 semantics, from an FP32 estimate E32 whose
// relative error is at most `bnd`; falls back to the FP64 definition.
__device__ bool decide_pass(const MxArgs& a, MxSmem& S, const Geom& g, int r, double E32, double bnd, double el2,
                            double delta, float inv_delta, float delta_f) {
  // every thread evaluates the same expression on the same shared values
  const double lo = E32 / (1.0 + bnd), hi = E32 / (1.0 - bnd);
  if (hi < el2 * (1.0 - 1e-12)) return true;
  if (lo > el2 * (1.0 + 1e-12)) return false;
  if (threadIdx.x == 0) S.nexact += 1;
  const double E = exact_error(a, S, g, r, delta, inv_delta, delta_f);
  return E <= el2;
}


// ---------------------------------------------------------------- pass 1: Gram + statistics
// Two thread groups of 128; group g accumulates packed pairs [68g, 68g+68) over
// every row; group 0 also gathers the block statistics.
// With `project`, the rows are first projected onto the current basis S.Vst
// (x <- x Vst) and the statistics are skipped: this accumulates the
// Rayleigh-Ritz matrix Vst^T G Vst, whose FP32 rounding errors scale with
// sqrt(lambda_i lambda_j) instead of the largest eigenvalue.
__device__ void pass_gram(const MxArgs& a, MxSmem& S, const Geom& g, bool project) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / kGrp, gt = tid % kGrp;
  const int n = g.n;
  float acc[kHalf];
#pragma unroll
  for (int p = 0; p < kHalf; ++p) acc[p] = 0.0f;
  float mn = INFINITY, mx = -INFINITY, tg = 0.0f, xg = 0.0f, rowmax = 0.0f;
  double sum = 0.0;
  int bad = 0;
  // Warp-uniform trip count: every lane runs every iteration (rows past the
  // end load zeros and are masked out), so the shuffles below always see the
  // full warp.
  for (int64_t l0 = gt - lane; l0 < g.L; l0 += kGrp) {
    const int64_t l = l0 + lane;
    const bool valid = l < g.L;
    float x[NM];
    if (valid) load_row(a, S, g, l, x);
    else {
#pragma unroll
      for (int j = 0; j < NM; ++j) x[j] = 0.0f;
    }
    if (project) {
      float c[NM];
      const float a0 = x[0];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < NM; ++j)
          if (j < n && k < n) v = __fmaf_rn(__fsub_rn(x[j], a0), S.Vst[j * NM + k], v);
        c[k] = k < n ? __fmaf_rn(a0, S.vsum[k], v) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) x[k] = c[k];
    }
    if (grp == 0 && !project) {
#pragma unroll
      for (int i = 0, p = 0; i < NM; ++i)
#pragma unroll
        for (int j = i; j < NM; ++j, ++p)
          if (p < kHalf) acc[p] = __fmaf_rn(x[i], x[j], acc[p]);
      float rn = 0.0f;
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (j < n && valid) {
          const float v = x[j];
          if (!isfinite(v)) bad = 1;
          mn = fminf(mn, v);
          mx = fmaxf(mx, v);
          sum += (double)v;
          rn = __fmaf_rn(v, v, rn);
          if (j + 1 < n) { const float d = x[j + 1] - v; tg = __fmaf_rn(d, d, tg); }
        }
      }
      rowmax = fmaxf(rowmax, rn);
      // x-neighbour: next row of the warp when it is the next x in the same x-run
      const int64_t ls = l;
      const bool has_next = valid && (g.side == 0) && ((ls % g.sx) + 1 < g.sx) && (lane < 31) && (l + 1 < g.L);
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        const float nb = __shfl_down_sync(0xffffffffu, x[j], 1);
        if (has_next && j < n) { const float d = nb - x[j]; xg = __fmaf_rn(d, d, xg); }
      }
    } else if (grp == 0) {
#pragma unroll
      for (int i = 0, p = 0; i < NM; ++i)
#pragma unroll
        for (int j = i; j < NM; ++j, ++p)
          if (p < kHalf) acc[p] = __fmaf_rn(x[i], x[j], acc[p]);
    } else {
#pragma unroll
      for (int i = 0, p = 0; i < NM; ++i)
#pragma unroll
        for (int j = i; j < NM; ++j, ++p)
          if (p >= kHalf) acc[p - kHalf] = __fmaf_rn(x[i], x[j], acc[p - kHalf]);
    }
  }
  // fixed-order reduction: warp xor tree, then the 4 warps of the group in order
#pragma unroll
  for (int p = 0; p < kHalf; ++p) {
    float v = acc[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) S.red[warp][p] = v;
  }
  if (grp == 0 && !project) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      tg += __shfl_xor_sync(0xffffffffu, tg, o);
      xg += __shfl_xor_sync(0xffffffffu, xg, o);
      rowmax = fmaxf(rowmax, __shfl_xor_sync(0xffffffffu, rowmax, o));
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
      bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
      S.st_min[warp] = mn; S.st_max[warp] = mx; S.st_gt[warp] = tg; S.st_gx[warp] = xg;
      S.st_rowmax[warp] = rowmax; S.st_sum[warp] = sum;
      if (bad) S.nonfinite = 1;
    }
  }
  __syncthreads();
  if (tid < kNP) {
    const int gw = (tid / kHalf) * 4, pp = tid % kHalf;
    float v = 0.0f;
    for (int w = 0; w < 4; ++w) v = __fadd_rn(v, S.red[gw + w][pp]);
    int i = 0, rem = tid;
    while (rem >= NM - i) { rem -= NM - i; ++i; }
    const int j = i + rem;
    if (i < n && j < n) {
      S.G32[i * NM + j] = v; S.G32[j * NM + i] = v;
      S.G64[i * NM + j] = (double)v; S.G64[j * NM + i] = (double)v;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- encode pass
// Projection, quantization and decode at rank r; with `check`, FP32 estimates
// of E(r-1) and E(r) land in S.Ered[0], S.Ered[1].  Stores q (columns < r) in
// the CTA scratch, the corrections in k8/k32, widths and counts in S.
__device__ void pass_encode(const MxArgs& a, MxSmem& S, const Geom& g, int r, bool check, double delta,
                            float inv_delta, float delta_f, const CorrConst& cc, bool pointwise, int32_t* qs,
                            int8_t* k8, int32_t* k32) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int n = g.n;
  if (tid < NM) S.wq[tid] = 0;
  if (tid == 0) { S.kmax = 0; S.ncorr = 0; S.nesc = 0; }
  __syncthreads();
  float e1 = 0.0f, e2 = 0.0f;
  uint32_t qmx[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) qmx[k] = 0;
  int nc = 0, ne = 0;
  uint32_t kmx = 0;
  int ovf = 0;
  for (int64_t l = tid; l < g.L; l += kMT) {
    float x[NM];
    load_row(a, S, g, l, x);
    int32_t q[NM];
    float ch[NM];
    row_coeffs(S, x, n, r, delta, inv_delta, delta_f, q, ch, ovf);
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      if (k < r) {
        qs[(int64_t)k * g.L + l] = q[k];
        const uint32_t z = zigzag(q[k]);
        qmx[k] = z > qmx[k] ? z : qmx[k];
      }
    }
    float acc[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) acc[j] = 0.0f;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      if (k < r) {
        if (check && k == r - 1) {
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < n) { const float d = __fsub_rn(x[j], acc[j]); e1 = __fmaf_rn(d, d, e1); }
        }
#pragma unroll
        for (int j = 0; j < NM; ++j)
          if (j < n) acc[j] = __fmaf_rn(ch[k], S.Vst[j * NM + k], acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < NM; ++j) {
      if (j < n) {
        if (check) { const float d = __fsub_rn(x[j], acc[j]); e2 = __fmaf_rn(d, d, e2); }
        const int64_t e = a_elem(g, l, j);
        int32_t kv = 0;
        if (pointwise) kv = corr_exact(x[j], acc[j], cc);
        if (kv == kEscape) {
          ++ne;
          k8[e] = (int8_t)-128;
          k32[e] = kEscape;
        } else {
          if (kv != 0) {
            ++nc;
            const uint32_t z = zigzag(kv);
            kmx = z > kmx ? z : kmx;
          }
          if (kv >= -127 && kv <= 127) {
            k8[e] = (int8_t)kv;
          } else {
            k8[e] = (int8_t)-128;
            k32[e] = kv;
          }
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    kmx = max(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
    ovf |= __shfl_xor_sync(0xffffffffu, ovf, o);
  }
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    uint32_t v = qmx[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && k < r && v) atomicMax(&S.wq[k], bit_width(v));
  }
  if (lane == 0) {
    if (nc) atomicAdd(&S.ncorr, nc);
    if (ne) atomicAdd(&S.nesc, ne);
    if (kmx) atomicMax(&S.kmax, (int)kmx);
    if (ovf) S.ovf = 1;
  }
  float ev[2] = {e1, e2};
  if (check) cta_reduce_floats(S, ev, 2);
  else __syncthreads();
}

// ---------------------------------------------------------------- record into the staging slot
__device__ void write_record(const MxArgs& a, MxSmem& S, const Geom& g, int64_t bi, bool raw, int r,
                             const int32_t* qs, const int8_t* k8, const int32_t* k32) {
  const int tid = threadIdx.x;
  const int n = g.n;
  const int64_t L = g.L, N = g.N, M = g.M;
  uint8_t* rec = a.staging + align_up((g.pt_off - a.P.pt_base) * 4, 16) + 48 * bi;
  __shared__ BlockMeta m;
  __shared__ RecLayout lay;
  if (tid == 0) {
    const int64_t rawsz = raw_record_bytes(N, 4);
    m.rcap = a.P.rank_cap < n ? a.P.rank_cap : n;
    m.nprobes = 0;
    for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
    m.flags = g.side ? (int)kFlagSpatial : 0;
    m.r = 0; m.wk = 0; m.ib = 0; m.ncorr = 0; m.nesc = 0;
    bool israw = raw;
    if (!israw) {
      for (int k = 0; k < r; ++k) m.wq[k] = (uint8_t)S.wq[k];
      const int wk = bit_width((uint32_t)S.kmax);
      const int ib = bit_width((uint32_t)(N - 1));
      lay = rec_layout(r, n, L, N, 4, m.wq, wk, ib, S.ncorr, S.nesc);
      if (lay.size >= rawsz) {
        israw = true;
      } else {
        m.r = r; m.wk = wk; m.ib = ib; m.ncorr = S.ncorr; m.nesc = S.nesc;
        m.flags |= lay.dense ? (int)kFlagDense : 0;
        m.nbytes = lay.size;
      }
    }
    if (israw) {
      m.r = 0; m.wk = 0; m.ib = 0; m.ncorr = 0; m.nesc = 0;
      for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
      m.flags = (int)kFlagRaw | (g.side ? (int)kFlagSpatial : 0);
      m.nbytes = rawsz;
    }
    a.meta[bi] = m;
    if (a.ranks) a.ranks[bi] = (m.flags & kFlagRaw) ? -1 : m.r;
  }
  __syncthreads();
  for (int64_t i = tid; i < m.nbytes / 16; i += kMT) reinterpret_cast<uint4*>(rec)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  if (tid == 0) {
    rec[0] = (uint8_t)m.r;
    rec[1] = (uint8_t)m.flags;
    rec[2] = (uint8_t)m.wk;
    rec[3] = (uint8_t)m.ib;
    reinterpret_cast<uint32_t*>(rec)[1] = (uint32_t)m.ncorr;
    reinterpret_cast<uint32_t*>(rec)[2] = (uint32_t)m.nesc;
    reinterpret_cast<uint32_t*>(rec)[3] = (uint32_t)m.nbytes;
  }
  if (m.flags & kFlagRaw) {
    float* vals = reinterpret_cast<float*>(rec + 16);
    for (int64_t e = tid; e < N; e += kMT) {
      const int64_t lt = e / M, ls = e - lt * M;
      vals[e] = a.in[gidx(a, S, g, ls, lt)];
    }
    __syncthreads();
    return;
  }
  const int rr = m.r;
  for (int c = tid; c < rr; c += kMT) rec[lay.off_wq + c] = m.wq[c];
  float* vout = reinterpret_cast<float*>(rec + lay.off_v);
  for (int i = tid; i < n * rr; i += kMT) {
    const int c = i / n, j = i - c * n;
    vout[i] = S.Vst[j * NM + c];
  }
  uint32_t* qw = reinterpret_cast<uint32_t*>(rec + lay.off_q);
  // Each task packs 32 consecutive values of one stream; 32 values of w bits
  // are exactly w words, so tasks never share an output word.
  {
    int64_t wbase = 0;
    __shared__ int64_t colbase[NM + 1];
    if (tid == 0) {
      for (int c = 0; c < rr; ++c) { colbase[c] = wbase; wbase += (L * m.wq[c] + 31) / 32; }
      colbase[rr] = wbase;
    }
    __syncthreads();
    const int64_t runs = cdiv(L, 32);
    for (int64_t task = tid; task < runs * rr; task += kMT) {
      const int c = (int)(task / runs);
      const int64_t first = (task - (int64_t)c * runs) * 32;
      const int wdt = m.wq[c];
      if (wdt == 0) continue;
      const int32_t* col = qs + (int64_t)c * L + first;
      const int cnt = (int)((L - first) < 32 ? (L - first) : 32);
      int32_t v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = i < cnt ? col[i] : 0;
      uint32_t* dst = qw + colbase[c] + (first / 32) * wdt;
      uint64_t acc = 0;
      int nbits = 0, wo = 0;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (i < cnt) {
          acc |= (uint64_t)zigzag(v[i]) << nbits;
          nbits += wdt;
          if (nbits >= 32) { dst[wo++] = (uint32_t)acc; acc >>= 32; nbits -= 32; }
        }
      }
      if (nbits > 0) dst[wo] = (uint32_t)acc;
    }
  }
  auto kval = [&](int64_t e) -> int32_t {
    const int8_t v = k8[e];
    return v == (int8_t)-128 ? k32[e] : (int32_t)v;
  };
  uint32_t* cw = reinterpret_cast<uint32_t*>(rec + lay.off_c);
  if (m.wk > 0) {
    if (lay.dense) {
      const int wk = m.wk;
      const int64_t runs = cdiv(N, 32);
      for (int64_t task = tid; task < runs; task += kMT) {
        const int64_t first = task * 32;
        const int cnt = (int)((N - first) < 32 ? (N - first) : 32);
        int8_t kb[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) kb[i] = i < cnt ? k8[first + i] : (int8_t)0;
        uint32_t* dst = cw + task * wk;
        uint64_t acc = 0;
        int nbits = 0, wo = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (i < cnt) {
            int32_t kv = kb[i];
            if (kv == -128) kv = k32[first + i];
            acc |= (uint64_t)(kv == kEscape ? 0u : zigzag(kv)) << nbits;
            nbits += wk;
            if (nbits >= 32) { dst[wo++] = (uint32_t)acc; acc >>= 32; nbits -= 32; }
          }
        }
        if (nbits > 0) dst[wo] = (uint32_t)acc;
      }
    } else {
      __syncthreads();
      int base = 0;
      for (int64_t e0 = 0; e0 < N; e0 += kMT) {
        const int64_t e = e0 + tid;
        const int32_t kv = e < N ? kval(e) : 0;
        const int flag = (e < N && kv != 0 && kv != kEscape) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(flag, S.sh_warp, &tot);
        if (flag) {
          const uint64_t pos = (uint64_t)(base + ex) * (uint64_t)(m.ib + m.wk);
          or_bits(cw, pos, (uint32_t)e, m.ib);
          or_bits(cw, pos + m.ib, zigzag(kv), m.wk);
        }
        base += tot;
      }
    }
  }
  if (m.nesc > 0) {
    __syncthreads();
    uint32_t* ei = reinterpret_cast<uint32_t*>(rec + lay.off_ei);
    float* ev = reinterpret_cast<float*>(rec + lay.off_ev);
    int base = 0;
    for (int64_t e0 = 0; e0 < N; e0 += kMT) {
      const int64_t e = e0 + tid;
      const int flag = (e < N && k8[e] == (int8_t)-128 && k32[e] == kEscape) ? 1 : 0;
      int tot;
      const int ex = block_excl_scan(flag, S.sh_warp, &tot);
      if (flag) {
        ei[base + ex] = (uint32_t)e;
        const int64_t lt = e / M, ls = e - lt * M;
        ev[base + ex] = a.in[gidx(a, S, g, ls, lt)];
      }
      base += tot;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- rank prediction
// Warp 0: eigenvalue-tail rank estimate E(r) ~ sum_{i>=r} lambda_i + r L delta^2 / 12
// (truncation plus uniform quantization noise) and the 32 block features, one
// feature per lane in FP32 (the features only steer a prediction that is then
// checked exactly).
__device__ int predict_rank(const MxArgs& a, MxSmem& S, const Geom& g, int64_t bi, int rcap, double el2,
                            double delta, int lane) {
  const int n = g.n;
  // suffix sums tail[r] = sum_{i >= r} lambda_i by a warp scan (lane r)
  double t = lane < n ? S.lam[lane] : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_down_sync(0xffffffffu, t, o);
    if (lane + o < 32) t += y;
  }
  const double qn = (double)g.L * delta * delta / 12.0;
  const bool ok = lane <= rcap && (lane < n ? t : 0.0) + lane * qn <= el2;
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  const int rp = m ? (__ffs(m) - 1) : rcap;
  const double tot = __shfl_sync(0xffffffffu, t, 0);
  const double l0 = S.lam[0];
  float mn = S.st_min[0], mx = S.st_max[0], tg = 0.0f, xg = 0.0f;
  for (int w = 0; w < 4; ++w) {
    mn = fminf(mn, S.st_min[w]); mx = fmaxf(mx, S.st_max[w]);
    tg += S.st_gt[w]; xg += S.st_gx[w];
  }
  const float tot_f = (float)(tot > 0.0 ? tot : 1e-30);
  const float el2_f = (float)el2;
  float f = 0.0f;
  if (lane == 0) f = log10f(tot_f / el2_f + 1e-30f);
  // lanes 1..16: log10 of the tail beyond r = lane - 1
  const double tr = __shfl_sync(0xffffffffu, t, (lane - 1) & 31);
  if (lane >= 1 && lane <= 16) f = log10f((lane - 1 < n ? (float)tr : 0.0f) / el2_f + 1e-30f);
  if (lane >= 17 && lane <= 24) {
    const int i = lane - 16;
    f = (i < n && l0 > 0.0) ? sqrtf((float)(S.lam[i] / l0)) : 0.0f;
  }
  if (lane == 25) f = tg / tot_f;
  if (lane == 26) f = xg / tot_f;
  if (lane == 27) f = log10f((float)(qn / el2) + 1e-30f);
  if (lane == 28) f = log10f((float)(((double)mx - (double)mn) / delta) + 1e-30f);
  if (lane == 29) f = (float)((double)g.L * n / 65536.0);
  if (lane == 30) f = (float)n / 16.0f;
  if (lane == 31) f = (float)rp;
  S.featv[lane] = f;
  if (a.feat) a.feat[bi * kMlpF + lane] = f;
  return rp;
}

// ---------------------------------------------------------------- the persistent kernel
__device__ __forceinline__ void mixed_body(const MxArgs& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MxSmem& S = *reinterpret_cast<MxSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* qs = a.q_scr + (int64_t)blockIdx.x * NM * a.lmax;
  int8_t* k8 = a.k8_scr + (int64_t)blockIdx.x * a.nptmax;
  int32_t* k32 = a.k32_scr + (int64_t)blockIdx.x * a.nptmax;
  const Plan& P = a.P;
  if (tid == 0) { S.tab_sx = -1; S.tab_sy = -1; S.tab_sz = -1; S.tab_ok = 0; }
  unsigned long long ph[kPhases];
  for (int i = 0; i < kPhases; ++i) ph[i] = 0;
  long long tck = clock64();
  if (tid == 0) S.nexact = 0;
  auto mark = [&](int p) {
    const long long now = clock64();
    ph[p] += (unsigned long long)(now - tck);
    tck = now;
  };
  for (;;) {
    if (tid == 0) {
      int64_t b;
      for (;;) {
        b = (int64_t)atomicAdd(&a.status->pad[0], 1ull);
        if (b >= P.nb || !a.spatial_only || block_geom(P, P.b0 + b).side == 1) break;
      }
      S.bi = b;
    }
    __syncthreads();
    const int64_t bi = S.bi;
    if (bi >= P.nb) break;
    const Geom g = block_geom(P, P.b0 + bi);
    const VarInfo vi = a.vars[g.v];
    const int n = g.n;
    const int rcap = P.rank_cap < n ? P.rank_cap : n;
    const bool pointwise = P.eb_type != DLS_EB_NRMSE;
    const double delta = vi.delta;
    const float inv_delta = __double2float_rn(1.0 / delta), delta_f = __double2float_rn(delta);
    CorrConst cc;
    cc.eb = vi.eb;
    cc.step = vi.step;
    cc.step_f = __double2float_rn(vi.step);
    cc.inv_step_f = pointwise ? __double2float_rn(1.0 / vi.step) : 0.0f;
    cc.eb_lo_f = __double2float_rd(vi.eb * (1.0 - 1e-6));
    cc.eb_hi_f = __double2float_ru(vi.eb * (1.0 + 1e-6));
    const double el2 = (P.eb_type == DLS_EB_NRMSE) ? (vi.eb * vi.eb) * ((double)g.N / P.kbound)
                                                   : (vi.eb * vi.eb) * (double)g.N;
    if (tid == 0) { S.nonfinite = 0; S.ovf = 0; }
    prepare_block(a, S, g);

    tck = clock64();
    pass_gram(a, S, g, false);
    mark(kPhGram);
    if (S.nonfinite) {
      if (tid == 0) atomicOr(&a.status->nonfinite, 1u);
      __syncthreads();
      continue;
    }
    jacobi_cta<kMT>(S.G32, S.Vj, S.lam_t, n, 0.0f, S.jp);
    mark(kPhJacobi);
    {
      // FP64 copy of the Jacobi eigenvectors, then one orthonormalisation
      const int i = tid / NM, j = tid % NM;
      if (i < n && j < n) S.X64[i * NM + j] = (double)S.Vj[i * NM + j];
    }
    __syncthreads();
    reorth64(S, n);
    if (warp == 0) order_basis(S, n, lane);
    __syncthreads();
    mark(kPhRefine);
    // Tight bounds need the modes an FP32 Gram cannot resolve (eigenvalues near
    // 2^-24 trace G): one Rayleigh-Ritz step on the projected data fixes them.
    {
      double tr = 0.0;
      for (int i = 0; i < n; ++i) tr += S.lam[i];
      const double budget = (vi.eb * vi.eb) * (double)g.L;   // per-mode share of eps_l^2
      const double noise = (P.eb_type == DLS_EB_NRMSE ? el2 / n : budget);
      if (n > 1 && 4.0 * 5.9604644775390625e-8 * tr > 0.5 * noise) {
        pass_gram(a, S, g, true);
        jacobi_cta<kMT>(S.G32, S.Vj, S.lam_t, n, 0.0f, S.jp);
        // V = Vst W in FP64, eigenvalues from the rotated diagonal
        {
          const int i = tid / NM, j = tid % NM;
          if (i < n && j < n) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v = fma((double)S.Vst[i * NM + k], (double)S.Vj[k * NM + j], v);
            S.X64[i * NM + j] = v;
          }
        }
        __syncthreads();
        reorth64(S, n);
        if (warp == 0) order_basis(S, n, lane);
        __syncthreads();
      }
    }
    mark(kPhRR);

    // overflow guard: |c_k| <= ||row|| (1 + 1e-5) for every column
    float rowmax = 0.0f;
    for (int w = 0; w < 4; ++w) rowmax = fmaxf(rowmax, S.st_rowmax[w]);
    const bool may_overflow = !((double)sqrtf(rowmax) * 1.0001 / delta < 16777216.0 * 0.999);

    if (warp == 0) {
      const int rp = predict_rank(a, S, g, bi, rcap, el2, delta, lane);
      if (lane == 0) S.r_pred = rp;
    }
    __syncthreads();
    if (a.learned == kRankMlp && warp == 0) {
      const int rm = mlp_rank_warp(&g_rank_model, S.featv, S.mh1, lane, rcap);
      if (lane == 0) S.r_pred = rm;
    }
    __syncthreads();
    mark(kPhPredict);

    // error bound of the FP32 estimates of E(r)
    const int64_t rows_per_thread = cdiv(g.L, kMT);
    const double bnd = (double)(rows_per_thread * n + 40) * 6.6e-8;
    bool accepted = false;
    int r = 0;
    if (a.learned != kRankSearch && !may_overflow) {
      const int rp = S.r_pred;
      pass_encode(a, S, g, rp, true, delta, inv_delta, delta_f, cc, pointwise, qs, k8, k32);
      mark(kPhEncode);
      const double E_rm1 = S.Ered[0], E_r = S.Ered[1];
      if (!S.ovf) {
        const bool p_r = decide_pass(a, S, g, rp, E_r, bnd, el2, delta, inv_delta, delta_f);
        bool p_rm1 = false;
        if (rp > 0 && p_r) p_rm1 = decide_pass(a, S, g, rp - 1, E_rm1, bnd, el2, delta, inv_delta, delta_f);
        accepted = p_r && !p_rm1;
        r = rp;
      }
      mark(kPhDecide);
    }
    bool raw = false;
    if (!accepted) {
      // every warp has read S.ovf (above) before thread 0 clears it, so that
      // all take the same decision path and meet at the same barriers
      __syncthreads();
      if (tid == 0) S.ovf = 0;
      __syncthreads();
      int ovf = 0;
      pass_all_errors(a, S, g, rcap, delta, inv_delta, delta_f, ovf);
      if (ovf) S.ovf = 1;
      __syncthreads();
      double Eall[NM + 1];
      for (int i = 0; i <= rcap; ++i) Eall[i] = S.Ered[i];
      if (S.ovf) {
        raw = true;
      } else {
        int lo = 0, hi = rcap;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (decide_pass(a, S, g, mid, Eall[mid], bnd, el2, delta, inv_delta, delta_f)) hi = mid;
          else lo = mid + 1;
        }
        r = lo;
        if (!pointwise && !decide_pass(a, S, g, r, Eall[r], bnd, el2, delta, inv_delta, delta_f)) raw = true;
        if (!raw) pass_encode(a, S, g, r, false, delta, inv_delta, delta_f, cc, pointwise, qs, k8, k32);
      }
      mark(kPhSearch);
    }
    write_record(a, S, g, bi, raw, r, qs, k8, k32);
    mark(kPhPack);
    ph[accepted ? kCntAccepted : kCntSearched] += 1;
  }
  ph[kCntExact] = S.nexact;
  if (tid == 0 && a.phase)
    for (int i = 0; i < kPhases; ++i) a.phase[(int64_t)blockIdx.x * kPhases + i] += ph[i];
}

// Two occupancy variants of the same kernel: 2 CTAs per SM (128 registers per
// thread) or 1 CTA per SM (no register cap); a plan's tuning picks one as the
// form of the shape class this kernel serves with k_tile (the blocks that are
// not whole blocks of the encode pass).
template <int MINB>
__global__ void __launch_bounds__(kMT, MINB) k_mixed(MxArgs a) {
  mixed_body(a);
}

// Copies the staged records to their stream positions (deferred records are
// written there by the deferred packer instead).
__global__ void __launch_bounds__(256) k_compact(Plan P, const uint8_t* staging, const BlockMeta* meta,
                                                 const unsigned long long* offsets, Status* st, uint8_t* out) {
  if (st->capacity || st->nonfinite) return;
  for (int64_t bi = blockIdx.x; bi < P.nb; bi += gridDim.x) {
    if (meta[bi].flags & kFlagDeferred) continue;
    const Geom g = block_geom(P, P.b0 + bi);
    const uint4* src = reinterpret_cast<const uint4*>(staging + align_up((g.pt_off - P.pt_base) * 4, 16) + 48 * bi);
    uint4* dst = reinterpret_cast<uint4*>(out + P.payload_pos + offsets[bi]);
    const int64_t words = meta[bi].nbytes / 16;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
}

__global__ void k_stage_quantize(const float* c, int64_t n, double delta, int32_t* q, int32_t* ovf) {
  const float inv = __double2float_rn(1.0 / delta);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int o = 0;
    q[i] = quant_exact(c[i], delta, inv, o);
    ovf[i] = o;
  }
}

// path 0: corr_exact (the row-loading kernel's decision); 1: the per-block
// kernel's candidate filter, then corr_decide for candidates (its sparse
// encode pass); 2: corr_decide for every element (its dense encode pass).
__global__ void k_stage_correct(const float* x, const float* xh, int64_t n, double eb, int path, int32_t* k) {
  const CorrConst cc = make_corr_const(eb, 2.0 * eb, true);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float xi = x[i], hi = xh[i];
    if (path == 0) k[i] = corr_exact(xi, hi, cc);
    else if (path == 1) k[i] = corr_candidate(__fsub_rn(xi, hi), cc) ? corr_decide(xi, hi, cc) : 0;
    else k[i] = corr_decide(xi, hi, cc);
  }
}

}  // namespace

int launch_stage_quantize(const float* c, int64_t n, double delta, int32_t* q, int32_t* ovf, cudaStream_t s) {
  if (n <= 0) return DLS_OK;
  k_stage_quantize<<<(unsigned)(n < 65536 * 256 ? cdiv(n, 256) : 65536), 256, 0, s>>>(c, n, delta, q, ovf);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_stage_correct(const float* x, const float* xh, int64_t n, double eb, int path, int32_t* k,
                         cudaStream_t s) {
  if (n <= 0) return DLS_OK;
  k_stage_correct<<<(unsigned)(n < 65536 * 256 ? cdiv(n, 256) : 65536), 256, 0, s>>>(x, xh, n, eb, path, k);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

size_t mixed_smem_bytes() { return sizeof(MxSmem); }

namespace {
std::mutex g_model_mu;
bool g_model_loaded[64] = {};
}  // namespace

const MlpModel* rank_model_device() {
  void* p = nullptr;
  if (!rank_model_loaded() || cudaGetSymbolAddress(&p, g_rank_model) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return reinterpret_cast<const MlpModel*>(p);
}

bool rank_model_loaded() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lock(g_model_mu);
  return g_model_loaded[dev];
}

}  // namespace dls

extern "C" int dls_set_rank_model(const float* h_params, size_t count) {
  using namespace dls;
  if (!h_params || count != (size_t)kMlpNParam) return DLS_ERR_INVALID_ARG;
  for (size_t i = 0; i < count; ++i)
    if (!isfinite(h_params[i])) return DLS_ERR_INVALID_ARG;
  for (int f = 0; f < kMlpF; ++f)
    if (!(h_params[kMlpOffSig + f] > 0.0f)) return DLS_ERR_INVALID_ARG;
  MlpModel m;
  for (int f = 0; f < kMlpF; ++f) { m.mu[f] = h_params[kMlpOffMu + f]; m.sig[f] = h_params[kMlpOffSig + f]; }
  auto r = [](float x) { return __bfloat162float(__float2bfloat16_rn(x)); };
  for (int h = 0; h < kMlpH; ++h) {
    m.b1[h] = r(h_params[kMlpOffB1 + h]);
    m.b2[h] = r(h_params[kMlpOffB2 + h]);
    m.W3[h] = r(h_params[kMlpOffW3 + h]);
  }
  m.b3 = r(h_params[kMlpOffB3]);
  for (int h = 0; h < kMlpH; ++h) {
    for (int f = 0; f < kMlpF; ++f) m.W1t[f * kMlpH + h] = __float2bfloat16_rn(h_params[kMlpOffW1 + h * kMlpF + f]);
    for (int k = 0; k < kMlpH; ++k) m.W2t[k * kMlpH + h] = __float2bfloat16_rn(h_params[kMlpOffW2 + h * kMlpH + k]);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DLS_ERR_CUDA;
  if (cudaMemcpyToSymbol(g_rank_model, &m, sizeof(m)) != cudaSuccess) return DLS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_model_mu);
  g_model_loaded[dev] = true;
  return DLS_OK;
}

namespace dls {

int launch_mixed_compress(const Plan& p, const void* d_in, const MixedWork& w, int learned, int variant,
                          int spatial_only, cudaStream_t s) {
  if (p.nb == 0) return DLS_OK;
  MxArgs a;
  a.spatial_only = spatial_only;
  a.P = p;
  a.in = (const float*)d_in;
  a.staging = w.staging;
  a.meta = w.meta;
  a.vars = w.vars;
  a.status = w.status;
  a.q_scr = w.q_scr;
  a.k8_scr = w.k8_scr;
  a.k32_scr = w.k32_scr;
  a.feat = w.feat;
  a.ranks = w.ranks;
  a.lmax = w.lmax;
  a.nptmax = w.nptmax;
  a.learned = learned;
  a.phase = w.phase;
  const size_t smem = sizeof(MxSmem);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DLS_ERR_CUDA;
  int ctas = variant == 1 ? sms : 2 * sms;
  if (ctas > w.ctas) ctas = w.ctas;
  const int grid = (int)(p.nb < ctas ? p.nb : ctas);
  if (variant == 1) {
    if (cudaFuncSetAttribute(k_mixed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return DLS_ERR_CUDA;
    k_mixed<1><<<grid, kMT, smem, s>>>(a);
  } else {
    if (cudaFuncSetAttribute(k_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return DLS_ERR_CUDA;
    k_mixed<2><<<grid, kMT, smem, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_compact(const Plan& p, const MixedWork& w, void* d_out, cudaStream_t s) {
  if (p.nb == 0) return DLS_OK;
  const int grid = (int)(p.nb < 4096 ? p.nb : 4096);
  k_compact<<<grid, 256, 0, s>>>(p, w.staging, w.meta, w.offsets, w.status, (uint8_t*)d_out);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

}  // namespace dls
