// Device pieces shared by the two mixed-precision kernels (k_mixed.cu: row
// loader, any block side; k_tile.cu: staged tiles, time-side blocks):
// the FP64-semantics decisions behind FP32 filters, the rank-model layout and
// evaluation, and the register-resident Jacobi eigensolver.
#pragma once

#include <cuda_bf16.h>

#include "dls_device.cuh"

namespace dls {

constexpr int NM = 16;                   // largest Gram order on the mixed paths
constexpr float kTwo24 = 16777216.0f;

// ---------------------------------------------------------------- exact decisions
// q = rint((double)c / delta) with ties to even; *ovf when |c / delta| >= 2^24.
// The FP32 quotient decides whenever its distance to the nearest half-integer
// exceeds its rounding error (a few ulps of |y|); otherwise the FP64 quotient
// of the same c decides, so the result equals the FP64 definition.
// The FP64 branch is rare and kept out of line, so the unrolled callers stay small.
static __device__ __noinline__ int32_t quant_fp64(float c, double delta, int* ovf) {
  const double Y = __ddiv_rn((double)c, delta);
  if (!(fabs(Y) < 16777216.0)) { *ovf = 1; return 0; }
  return (int32_t)rint(Y);
}
__device__ __forceinline__ int32_t quant_exact(float c, double delta, float inv_delta, int& ovf) {
  const float y = __fmul_rn(c, inv_delta);
  const float ay = fabsf(y);
  const float m = __fmul_rn(ay, 4.0e-7f) + 1.0e-30f;   // > 3 * 2^-24 |y| + FP64 rounding
  const float r = rintf(y);
  const float fr = fabsf(__fsub_rn(y, r));
  if (fr < 0.5f - m && ay < kTwo24 * 0.999999f) return (int32_t)r;
  return quant_fp64(c, delta, &ovf);
}

struct CorrConst {
  double eb, step;
  float step_f, inv_step_f, eb_lo_f, eb_hi_f;
};

__host__ __device__ inline CorrConst make_corr_const(double eb, double step, bool pointwise) {
  CorrConst cc;
  cc.eb = eb;
  cc.step = step;
#ifdef __CUDA_ARCH__
  cc.step_f = __double2float_rn(step);
  cc.inv_step_f = pointwise ? __double2float_rn(1.0 / step) : 0.0f;
  cc.eb_lo_f = __double2float_rd(eb * (1.0 - 1e-6));
  cc.eb_hi_f = __double2float_ru(eb * (1.0 + 1e-6));
#else
  cc.step_f = (float)step;
  cc.inv_step_f = pointwise ? (float)(1.0 / step) : 0.0f;
  cc.eb_lo_f = 0.0f;
  cc.eb_hi_f = 0.0f;
#endif
  return cc;
}

// Pointwise correction with the FP64 definition (k = rint((x - xhat) / step),
// xt = fma(k, step, xhat) in float, escape when |x - xt| > eb or |k| > 2^20):
// returns k (0 if none) or kEscape.
static __device__ __noinline__ int32_t corr_slow(float x, float xh, const CorrConst& cc);
__device__ __forceinline__ int32_t corr_exact(float x, float xh, const CorrConst& cc) {
  const float R = __fsub_rn(x, xh);
  // |fl(x - xhat)| < eb (1 - 1e-6), rounded down, proves |x - xhat| < eb: k = 0, in bound
  if (fabsf(R) < cc.eb_lo_f) return 0;
  const float y = __fmul_rn(R, cc.inv_step_f);
  const float ay = fabsf(y);
  const float m = __fmul_rn(ay, 5.0e-7f) + 1.0e-30f;
  if (ay < 0.5f - m) return 0;            // |x - xhat| < eb certainly: k = 0, in bound
  // k from the FP32 quotient when it is clear of a half-integer and within
  // 2^20; the bound check in FP32 when clear of eb; anything else (ties,
  // escapes, the narrow band around eb) takes the full path out of line
  const float r = rintf(y);
  const float fr = fabsf(__fsub_rn(y, r));
  if (!(fr < 0.5f - m) || !(fabsf(r) <= 1048576.0f)) return corr_slow(x, xh, cc);
  const float xt = __fmaf_rn(r, cc.step_f, xh);
  const float d = fabsf(__fsub_rn(x, xt));
  if (d <= cc.eb_lo_f) return (int32_t)r;
  if (d >= cc.eb_hi_f) return kEscape;
  return corr_slow(x, xh, cc);
}
// The same decision without branches, for loops that decide many elements:
// returns k when the FP32 evaluation settles it, and sets *unsure otherwise
// (the caller then takes corr_slow, which decides with the FP64 definition).
__device__ __forceinline__ int32_t corr_fast(float x, float xh, const CorrConst& cc, bool* unsure) {
  const float R = __fsub_rn(x, xh);
  const bool zero = fabsf(R) < cc.eb_lo_f;           // |x - xhat| < eb certainly
  const float y = __fmul_rn(R, cc.inv_step_f);
  const float m = __fmul_rn(fabsf(y), 5.0e-7f) + 1.0e-30f;
  const float r = rintf(y);
  const bool clear = fabsf(__fsub_rn(y, r)) < 0.5f - m && fabsf(r) <= 1048576.0f;
  const float d = fabsf(__fsub_rn(x, __fmaf_rn(r, cc.step_f, xh)));
  const bool in = d <= cc.eb_lo_f, out = d >= cc.eb_hi_f;
  *unsure = !zero && !(clear && (in || out));
  return zero ? 0 : (out ? kEscape : (int32_t)r);
}
// The decision of one element the per-block kernel selected as a candidate
// (|fl(x - xhat)| at or above eb, rounded down): the branch-free FP32 test,
// and the FP64 definition where that test leaves the decision open.
static __device__ __noinline__ int32_t corr_slow(float x, float xh, const CorrConst& cc);
__device__ __forceinline__ int32_t corr_decide(float x, float xh, const CorrConst& cc) {
  bool u;
  const int32_t k = corr_fast(x, xh, cc, &u);
  return u ? corr_slow(x, xh, cc) : k;
}
// The candidate filter of the per-block kernel: elements with |fl(x - xhat)|
// below eb (1 - 1e-6), rounded down, need no correction and no decision.
__device__ __forceinline__ bool corr_candidate(float R, const CorrConst& cc) { return !(fabsf(R) < cc.eb_lo_f); }
static __device__ __noinline__ int32_t corr_slow(float x, float xh, const CorrConst& cc) {
  const float R = __fsub_rn(x, xh);
  const float y = __fmul_rn(R, cc.inv_step_f);
  const float ay = fabsf(y);
  const float m = __fmul_rn(ay, 5.0e-7f) + 1.0e-30f;
  double kk;
  const float r = rintf(y);
  const float fr = fabsf(__fsub_rn(y, r));
  if (fr < 0.5f - m) kk = (double)r;
  else kk = rint(__ddiv_rn(__dsub_rn((double)x, (double)xh), cc.step));
  float xt;
  if (kk == 0.0) {
    xt = xh;
  } else {
    if (fabs(kk) > kKmax) return kEscape;
    xt = __fmaf_rn((float)kk, cc.step_f, xh);
  }
  const float d = fabsf(__fsub_rn(x, xt));
  bool ok;
  if (d <= cc.eb_lo_f) ok = true;
  else if (d >= cc.eb_hi_f) ok = false;
  else ok = !(fabs(__dsub_rn((double)x, (double)xt)) > cc.eb);
  if (!ok) return kEscape;
  return (int32_t)kk;
}

// ---------------------------------------------------------------- rank model
// The trained block-rank MLP as the kernels read it (set by dls_set_rank_model).
// The two hidden layers' weights are stored transposed (W1t[f * kMlpH + h] =
// W1[h][f], W2t[k * kMlpH + h] = W2[h][k]) so that the 32 lanes of a warp, one
// output h each, read 64 consecutive bytes per input index.
struct MlpModel {
  float mu[kMlpF], sig[kMlpF];
  float b1[kMlpH], b2[kMlpH], W3[kMlpH], b3;
  __nv_bfloat16 W1t[kMlpF * kMlpH], W2t[kMlpH * kMlpH];
};

// Device copy of the model for the current device (null if none was set).
const MlpModel* rank_model_device();

// MLP prediction from the 32 features `featv` (shared) by one warp; h1 is a
// shared scratch of kMlpH floats.  BF16 weights, FP32 accumulation.
__device__ __forceinline__ int mlp_rank_warp(const MlpModel* M, const float* featv, float* h1, int lane, int rcap) {
  float z = 0.0f;
  if (lane < kMlpF) z = (featv[lane] - M->mu[lane]) / M->sig[lane];
  for (int hh = 0; hh < 2; ++hh) {
    const int h = lane + 32 * hh;
    float acc = M->b1[h];
#pragma unroll 8
    for (int f = 0; f < kMlpF; ++f)
      acc = fmaf(__bfloat162float(M->W1t[f * kMlpH + h]), __shfl_sync(0xffffffffu, z, f), acc);
    h1[h] = acc > 0.0f ? acc : 0.0f;
  }
  __syncwarp();
  float out = 0.0f;
  for (int hh = 0; hh < 2; ++hh) {
    const int h = lane + 32 * hh;
    float acc = M->b2[h];
#pragma unroll 8
    for (int k = 0; k < kMlpH; ++k) acc = fmaf(__bfloat162float(M->W2t[k * kMlpH + h]), h1[k], acc);
    acc = acc > 0.0f ? acc : 0.0f;
    out = fmaf(M->W3[h], acc, out);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
  out += M->b3;
  int r = (int)rintf(out);
  r = r < 0 ? 0 : (r > rcap ? rcap : r);
  __syncwarp();
  return r;
}

// ---------------------------------------------------------------- register Jacobi
template <int NP>
__device__ __forceinline__ float pick(const float (&a)[NP], int i) {
  float v = a[0];
#pragma unroll
  for (int j = 1; j < NP; ++j) v = (i == j) ? a[j] : v;
  return v;
}

// Parallel cyclic Jacobi of the symmetric matrix G (order n <= NP, row stride
// ldg, shared) by one warp, in FP32.  Lanes [0, NP) hold the rows of A by
// position, lanes [NP, 2 NP) the rows of the accumulated rotation V.  Each
// round rotates the position pairs (2k, 2k+1) at once; then rows and columns
// move one step along the round-robin circle (position 0 fixed), so NP - 1
// rounds pair every two positions once.  The permutation of the columns is
// fixed, so it is a renaming of registers.  Pairs with |a_pq| at or below the
// threshold are skipped: tol_abs, or with `relative` max(1e-7 sqrt(a_pp a_qq),
// 4 u max(a_pp, a_qq)) (reachable in FP32 on graded matrices), and never
// below floor_abs.  Stops after a
// sweep without rotation, or 30 sweeps.  Writes the eigenvectors as columns
// of Vout (row stride ldv) and the eigenvalues to lam, both in the original
// index order of the positions (any order: the caller sorts).
template <int NP>
__device__ void jacobi_reg(const float* G, int ldg, int n, bool relative, float tol_rel_trace, float* Vout, int ldv,
                           double* lam, int lane, float floor_abs = 0.0f) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int H = NP / 2;
  const bool isA = lane < NP;
  const bool isV = lane >= NP && lane < 2 * NP;
  const int row = isA ? lane : (isV ? lane - NP : 0);
  float a[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float v = 0.0f;
    if (isA) v = (row < n && j < n) ? G[row * ldg + j] : 0.0f;
    else if (isV) v = (row == j) ? 1.0f : 0.0f;
    a[j] = v;
  }
  int idx = row;
  float tr = (isA && row < n) ? pick<NP>(a, row) : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(FULL, tr, o);
  const float tol = tol_rel_trace * tr;
  const bool top = (row & 1) == 0;
  // source lane of the row moved into this position after a round
  int src = lane;
  if (isA) {
    if (row == 0) src = 0;
    else if (row == 2) src = 1;
    else if (!(row & 1)) src = row - 2;
    else if (row == NP - 1) src = NP - 2;
    else src = row + 2;
  }
  for (int sweep = 0; sweep < 30 && n > 1; ++sweep) {
    unsigned any = 0;
#pragma unroll 1
    for (int round = 0; round < NP - 1; ++round) {
      const float dself = pick<NP>(a, row);
      const float off = pick<NP>(a, row ^ 1);
      const float dpart = __shfl_xor_sync(FULL, dself, 1);
      const float apq = __shfl_sync(FULL, off, lane & ~1);
      const float app = top ? dself : dpart, aqq = top ? dpart : dself;
      float c = 1.0f, s = 0.0f, t = 0.0f;
      bool act = false;
      if (isA) {
        const float gpp = fabsf(app), gqq = fabsf(aqq);
        float thr = relative ? fmaxf(1.0e-7f * sqrtf(gpp * gqq), 4.0f * 5.9604645e-8f * fmaxf(gpp, gqq)) : tol;
        thr = fmaxf(thr, floor_abs);
        if (fabsf(apq) > thr && apq != 0.0f) {
          const float theta = (aqq - app) / (2.0f * apq);
          if (fabsf(theta) > 1e18f) t = 0.5f / theta;
          else t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(1.0f + theta * theta));
          c = 1.0f / sqrtf(1.0f + t * t);
          s = t * c;
          act = true;
        }
      }
      const unsigned actm = __ballot_sync(FULL, act);
      any |= actm;
      if (actm) {
        // columns (A and V lanes): a[:, 2k], a[:, 2k+1] rotated by pair k
#pragma unroll
        for (int k = 0; k < H; ++k) {
          const float ck = __shfl_sync(FULL, c, 2 * k), sk = __shfl_sync(FULL, s, 2 * k);
          const float x = a[2 * k], y = a[2 * k + 1];
          a[2 * k] = ck * x - sk * y;
          a[2 * k + 1] = sk * x + ck * y;
        }
        // rows (A lanes): this row with its partner's
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const float b = __shfl_xor_sync(FULL, a[j], 1);
          if (isA) a[j] = top ? (c * a[j] - s * b) : (s * b + c * a[j]);
        }
        // exact 2x2 result of the active pairs
        if (act) {
          const float nd = top ? app - t * apq : aqq + t * apq;
#pragma unroll
          for (int j = 0; j < NP; ++j) a[j] = (j == row) ? nd : ((j == (row ^ 1)) ? 0.0f : a[j]);
        }
      }
      // one step along the circle: rows between lanes, columns between registers
#pragma unroll
      for (int j = 0; j < NP; ++j) a[j] = __shfl_sync(FULL, a[j], src);
      idx = __shfl_sync(FULL, idx, src);
      float na[NP];
      na[0] = a[0];
      na[2] = a[1];
#pragma unroll
      for (int k = 2; k < H; ++k) na[2 * k] = a[2 * k - 2];
      na[NP - 1] = a[NP - 2];
#pragma unroll
      for (int k = 0; k + 1 < H; ++k) na[2 * k + 1] = a[2 * k + 3];
#pragma unroll
      for (int j = 0; j < NP; ++j) a[j] = na[j];
    }
    if (!any) break;
  }
  // eigenvalues (A lanes) and eigenvector columns (V lanes), by original index
  if (isA && idx < n) lam[idx] = (double)pick<NP>(a, row);
#pragma unroll
  for (int P = 0; P < NP; ++P) {
    const int ip = __shfl_sync(FULL, idx, P);
    if (isV && row < n && ip < n) Vout[row * ldv + ip] = a[P];
  }
  __syncwarp();
}

// ---------------------------------------------------------------- CTA Jacobi
// Scratch of the CTA Jacobi (shared).
struct JacPairs {
  int pq[NM / 2];                  // p | q << 8 | active << 16
  float2 cs[NM / 2];               // (c, s)
  float4 dg[NM / 2];               // (t, a_pp, a_qq, a_pq) for the exact 2x2 result
};

// Pair i of round `round` of the round-robin circle over m positions (m even).
__device__ __forceinline__ void circle_pair(int round, int i, int m, int& p, int& q) {
  int a, b;
  if (i == 0) { a = m - 1; b = round; }
  else { a = (round + i) % (m - 1); b = (round - i + (m - 1)) % (m - 1); }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Parallel cyclic Jacobi of the symmetric matrix A (order n <= NM, row stride
// NM, shared, overwritten) by all NT threads of the CTA, in FP32; V (shared)
// receives the eigenvectors as columns and lam the eigenvalues (diagonal),
// both by index.  Each round rotates m/2 disjoint pairs of the round-robin
// circle (m = n rounded up to even): rotation parameters by m/2 threads, then
// in one step every 2x2 block of A (rows of pair k, columns of pair l) becomes
// J_k^T A_kl J_l, with the exact 2x2 result on the rotated diagonal blocks, and
// the columns of V rotate.  Thresholds as in
// jacobi_reg (relative, with floor_abs).  Stops after a sweep without rotation
// or 30 sweeps.  All threads call.
template <int NT, int HF = 0>
__device__ void jacobi_cta(float* A, float* V, double* lam, int n, float floor_abs, JacPairs& J) {
  const int tid = threadIdx.x;
  const int m = HF ? 2 * HF : n + (n & 1);
  const int h = HF ? HF : m / 2;         // HF: the pair count at compile time (order 2 HF)
  for (int e = tid; e < NM * NM; e += NT) {
    const int i = e / NM, j = e % NM;
    V[e] = (i == j) ? 1.0f : 0.0f;
    if (i >= n || j >= n) A[e] = 0.0f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30 && n > 1; ++sweep) {
    int any = 0;
    for (int round = 0; round < m - 1; ++round) {
      int act = 0;
      if (tid < h) {
        int p, q;
        circle_pair(round, tid, m, p, q);
        const float app = A[p * NM + p], aqq = A[q * NM + q], apq = A[p * NM + q];
        const float gpp = fabsf(app), gqq = fabsf(aqq);
        const float thr = fmaxf(fmaxf(1.0e-7f * sqrtf(gpp * gqq), 4.0f * 5.9604645e-8f * fmaxf(gpp, gqq)), floor_abs);
        float c = 1.0f, s = 0.0f, t = 0.0f;
        if (fabsf(apq) > thr && apq != 0.0f) {
          // approximate division and reciprocal square root: any rotation
          // within a few ulps of orthogonal will do, as the FP64 refinement
          // restores orthonormality
          const float theta = __fdividef(aqq - app, 2.0f * apq);
          if (fabsf(theta) > 1e18f) t = __fdividef(0.5f, theta);
          else t = __fdividef(theta >= 0.0f ? 1.0f : -1.0f, fabsf(theta) + __fsqrt_rn(1.0f + theta * theta));
          c = rsqrtf(1.0f + t * t);
          s = t * c;
          act = 1;
        }
        J.pq[tid] = p | q << 8 | act << 16;
        J.cs[tid] = make_float2(c, s);
        J.dg[tid] = make_float4(t, app, aqq, apq);
      }
      if (!__syncthreads_or(act)) continue;
      any = 1;
      // one step: every 2x2 block (pair k rows, pair l columns) of A becomes
      // J_k^T A_kl J_l (the exact 2x2 result on the rotated diagonal blocks),
      // and the two columns of every active pair of V rotate
      const int nblk = h * h;
      for (int it = tid; it < nblk + n * h; it += NT) {
        if (it < nblk) {
          const int k = it / h, l = it - k * h;
          const int jk = J.pq[k], jl = J.pq[l];
          if (!((jk | jl) >> 16)) continue;
          const int p = jk & 255, q = (jk >> 8) & 255, pp = jl & 255, qq = (jl >> 8) & 255;
          const float2 csk = J.cs[k], csl = J.cs[l];
          const float ck = csk.x, sk = csk.y, cl = csl.x, sl = csl.y;
          const float a = A[p * NM + pp], b = A[p * NM + qq], c = A[q * NM + pp], d = A[q * NM + qq];
          const float r1 = ck * a - sk * c, r2 = ck * b - sk * d, r3 = sk * a + ck * c, r4 = sk * b + ck * d;
          float na = cl * r1 - sl * r2, nb = sl * r1 + cl * r2, nc = cl * r3 - sl * r4, nd = sl * r3 + cl * r4;
          if (k == l) {
            const float4 dg = J.dg[k];      // (t, a_pp, a_qq, a_pq)
            na = dg.y - dg.x * dg.w;
            nb = 0.0f;
            nc = 0.0f;
            nd = dg.z + dg.x * dg.w;
          }
          A[p * NM + pp] = na;
          A[p * NM + qq] = nb;
          A[q * NM + pp] = nc;
          A[q * NM + qq] = nd;
        } else {
          const int it2 = it - nblk;
          const int i = it2 / h, l = it2 - i * h;
          const int jl = J.pq[l];
          if (!(jl >> 16)) continue;
          const int p = jl & 255, q = (jl >> 8) & 255;
          const float2 csl = J.cs[l];
          const float c = csl.x, sv = csl.y;
          const float x = V[i * NM + p], y = V[i * NM + q];
          V[i * NM + p] = c * x - sv * y;
          V[i * NM + q] = sv * x + c * y;
        }
      }
      __syncthreads();
    }
    if (!any) break;
    // after a sweep with rotations: stop if no pair is above its threshold
    // now (the next sweep would rotate nothing), instead of running it
    int above = 0;
    for (int t = tid; t < n * (n - 1) / 2; t += NT) {
      int i = 0, rem = t;
      while (rem >= n - 1 - i) { rem -= n - 1 - i; ++i; }
      const int j = i + 1 + rem;
      const float app = A[i * NM + i], aqq = A[j * NM + j], apq = A[i * NM + j];
      const float gpp = fabsf(app), gqq = fabsf(aqq);
      const float thr = fmaxf(fmaxf(1.0e-7f * sqrtf(gpp * gqq), 4.0f * 5.9604645e-8f * fmaxf(gpp, gqq)), floor_abs);
      if (fabsf(apq) > thr && apq != 0.0f) above = 1;
    }
    if (!__syncthreads_or(above)) break;
  }
  if (tid < n) lam[tid] = (double)A[tid * NM + tid];
  __syncthreads();
}

}  // namespace dls
