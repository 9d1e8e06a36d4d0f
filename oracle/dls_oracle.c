/*
 * dls_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.  Every step is
 * written for a reader to check against the paper by eye; nothing here is
 * blocked, fused or reordered beyond what the definitions below state.
 *
 * Built with -O2 -fno-fast-math -ffp-contract=off: every a*b+c is two
 * roundings unless fma() is written out.
 *
 * Paper references are to arXiv 2601.20113 (section / equation / algorithm).
 */
#include "dls_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Stream format constants (an interface both sides implement).        */
/* ------------------------------------------------------------------ */
#define OR_MAGIC 0x31534C44u /* "DLS1" little endian */
#define OR_VERSION 1u
#define OR_HDR 128
#define OR_VARREC 32
#define OR_FLAG_RAW 1u
#define OR_FLAG_SPATIAL 2u
#define OR_FLAG_DENSE 4u
#define OR_FLAG_RICE 8u
#define OR_RICE_CHUNK 1024
#define OR_QMAX_F32 16777216.0    /* 2^24: |q| must stay below, so float(q) is exact */
#define OR_QMAX_F64 1073741824.0  /* 2^30 */
#define OR_KMAX 1048576.0         /* 2^20: larger corrections become escapes */

static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static int64_t al(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
static int esize(int dtype) { return dtype == OR_F32 ? 4 : 8; }

/* value x rounded to the field dtype, held in a double */
static double to_dt(double x, int dtype) { return dtype == OR_F32 ? (double)(float)x : x; }

static double field_at(const void* f, int dtype, int64_t i) {
  return dtype == OR_F32 ? (double)((const float*)f)[i] : ((const double*)f)[i];
}

/* ------------------------------------------------------------------ */
/* Block tiling (Algorithm 1, step 2: partition the domain into patches). */
/* Blocks tile x,y,z,t from the origin; edge blocks are truncated.       */
/* Block order: variable, then t, z, y, x block index (x fastest).       */
/* ------------------------------------------------------------------ */
int64_t or_num_blocks(const or_params* p) {
  int64_t nb = p->nvars;
  for (int a = 0; a < 4; ++a) nb *= cdiv(p->dims[a], p->block[a]);
  return nb;
}

int or_block_geom(const or_params* p, int64_t b, or_geom* g) {
  int64_t nbx = cdiv(p->dims[0], p->block[0]), nby = cdiv(p->dims[1], p->block[1]);
  int64_t nbz = cdiv(p->dims[2], p->block[2]), nbt = cdiv(p->dims[3], p->block[3]);
  int64_t ix = b % nbx; b /= nbx;
  int64_t iy = b % nby; b /= nby;
  int64_t iz = b % nbz; b /= nbz;
  int64_t it = b % nbt; b /= nbt;
  g->v = (int32_t)b;
  g->x0 = ix * p->block[0]; g->y0 = iy * p->block[1];
  g->z0 = iz * p->block[2]; g->t0 = it * p->block[3];
  g->sx = (int32_t)(p->dims[0] - g->x0 < p->block[0] ? p->dims[0] - g->x0 : p->block[0]);
  g->sy = (int32_t)(p->dims[1] - g->y0 < p->block[1] ? p->dims[1] - g->y0 : p->block[1]);
  g->sz = (int32_t)(p->dims[2] - g->z0 < p->block[2] ? p->dims[2] - g->z0 : p->block[2]);
  g->st = (int32_t)(p->dims[3] - g->t0 < p->block[3] ? p->dims[3] - g->t0 : p->block[3]);
  g->M = (int64_t)g->sx * g->sy * g->sz;
  g->T = g->st;
  g->N = g->M * g->T;
  /* Gram side: the smaller of space and time; time wins a tie. */
  if (g->T <= g->M) { g->side = 0; g->n = (int32_t)g->T; g->L = g->M; }
  else              { g->side = 1; g->n = (int32_t)g->M; g->L = g->T; }
  return 0;
}

int or_validate(const or_params* p) {
  if (!p || p->nvars < 1 || !p->eb) return OR_ERR_INVALID_ARG;
  if (p->dtype != OR_F32 && p->dtype != OR_F64) return OR_ERR_INVALID_ARG;
  if (p->eb_type < 0 || p->eb_type > 2) return OR_ERR_INVALID_ARG;
  if (p->rank_cap < 0) return OR_ERR_INVALID_ARG;
  for (int a = 0; a < 4; ++a)
    if (p->dims[a] < 1 || p->block[a] < 1 || p->block[a] > p->dims[a]) return OR_ERR_INVALID_ARG;
  int64_t M = (int64_t)p->block[0] * p->block[1] * p->block[2];
  int64_t T = p->block[3];
  if ((M < T ? M : T) > 32) return OR_ERR_INVALID_ARG;   /* Gram order n <= 32 */
  if (M * T > (1LL << 26)) return OR_ERR_INVALID_ARG;
  for (int v = 0; v < p->nvars; ++v)
    if (!(p->eb[v] > 0.0) || !isfinite(p->eb[v])) return OR_ERR_INVALID_ARG;
  int64_t nb = or_num_blocks(p);
  int64_t e = p->block_end < 0 ? nb : p->block_end;
  if (p->block_begin < 0 || p->block_begin > e || e > nb) return OR_ERR_INVALID_ARG;
  if (p->basis) {
    /* a fixed basis: order 1..32, finite, orthonormal columns to 1e-12 */
    int bn = p->basis_n;
    if (bn < 1 || bn > 32) return OR_ERR_INVALID_ARG;
    for (int i = 0; i < bn; ++i)
      for (int j = 0; j < bn; ++j) {
        double d = 0.0;
        for (int a = 0; a < bn; ++a) {
          if (!isfinite(p->basis[a * bn + i])) return OR_ERR_INVALID_ARG;
          d += p->basis[a * bn + i] * p->basis[a * bn + j];
        }
        if (fabs(d - (i == j ? 1.0 : 0.0)) > 1e-12) return OR_ERR_INVALID_ARG;
      }
  }
  if (p->global_stats) {
    /* whole-field statistics: finite, min <= max, sum >= 0, one point count
       (>= 1, integral) shared by every variable */
    const double pts = p->global_stats[3];
    for (int v = 0; v < p->nvars; ++v) {
      const double* g = p->global_stats + 4 * v;
      for (int i = 0; i < 4; ++i)
        if (!isfinite(g[i])) return OR_ERR_INVALID_ARG;
      if (!(g[0] <= g[1]) || g[2] < 0.0 || g[3] < 1.0 || g[3] != pts || g[3] != floor(g[3]))
        return OR_ERR_INVALID_ARG;
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Bound resolution (Sec. 2.4, Eq. 4).                                  */
/*   ABS:       eb as given                                              */
/*   REL_RANGE: eb = value * (max - min) of the variable                 */
/*   NRMSE:     eps = eps_t * ||u||_2 / 100 (paper's global L2 budget)   */
/* Quantization step delta: eb (pointwise modes) or eps/sqrt(K) (NRMSE). */
/* ------------------------------------------------------------------ */
int or_resolve(const or_params* p, const void* field, or_var* vars) {
  int64_t K = p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  for (int v = 0; v < p->nvars; ++v) {
    double mn = INFINITY, mx = -INFINITY, s2 = 0.0;
    for (int64_t i = 0; i < K; ++i) {
      double x = field_at(field, p->dtype, (int64_t)v * K + i);
      if (!isfinite(x)) return OR_ERR_NONFINITE;
      if (x < mn) mn = x;
      if (x > mx) mx = x;
      s2 = fma(x, x, s2);
    }
    int64_t Kb = K;
    if (p->global_stats) {
      /* the whole field's statistics replace the part's own */
      const double* g = p->global_stats + 4 * v;
      mn = g[0];
      mx = g[1];
      s2 = g[2];
      Kb = (int64_t)g[3];
    }
    or_var* o = &vars[v];
    o->eb_user = p->eb[v];
    o->K = Kb;
    o->norm2 = s2;
    if (p->eb_type == OR_EB_ABS) {
      o->eb = p->eb[v];
    } else if (p->eb_type == OR_EB_REL_RANGE) {
      double range = mx - mn;
      o->eb = range > 0.0 ? p->eb[v] * range : p->eb[v];
    } else {
      o->eb = p->eb[v] * sqrt(s2) / 100.0;
    }
    if (p->eb_type == OR_EB_NRMSE) {
      o->delta = o->eb > 0.0 ? o->eb / sqrt((double)Kb) : 1.0;
      o->step = 0.0;
    } else {
      o->delta = o->eb;
      o->step = 2.0 * o->eb;
    }
  }
  return OR_OK;
}

/* Squared local tolerance eps_l^2 for a block of N points (Sec. 2.4,
 * Eq. 4 with "patch size" = N and "number of coarsened elements" = K).
 *   pointwise modes: eps = eb*sqrt(K)  =>  eps_l^2 = eb^2 * N
 *   NRMSE:           eps_l^2 = eps^2 * (N / K)                          */
static double el2_of(const or_params* p, const or_var* o, int64_t N) {
  if (p->eb_type == OR_EB_NRMSE) return (o->eb * o->eb) * ((double)N / (double)o->K);
  return (o->eb * o->eb) * (double)N;
}

/* ------------------------------------------------------------------ */
/* Block data matrix.  Rows of the paper's sample matrix are patches;    */
/* here A (L x n) holds one block, long side as rows, Gram side as       */
/* columns.  Temporal side: A[l][j] = u(spatial l, time j).  Spatial     */
/* side: A[l][j] = u(spatial j, time l).  Spatial index is x fastest.    */
/* ------------------------------------------------------------------ */
void or_gather(const or_params* p, const void* field, const or_geom* g, double* A) {
  int64_t nx = p->dims[0], ny = p->dims[1], nz = p->dims[2];
  int64_t P = nx * ny * nz, base = (int64_t)g->v * P * p->dims[3];
  for (int32_t lt = 0; lt < g->st; ++lt)
    for (int32_t lz = 0; lz < g->sz; ++lz)
      for (int32_t ly = 0; ly < g->sy; ++ly)
        for (int32_t lx = 0; lx < g->sx; ++lx) {
          int64_t ls = ((int64_t)lz * g->sy + ly) * g->sx + lx;
          int64_t gi = base + (g->t0 + lt) * P + (g->z0 + lz) * nx * ny + (g->y0 + ly) * nx + (g->x0 + lx);
          double x = field_at(field, p->dtype, gi);
          if (g->side == 0) A[ls * g->n + lt] = x;
          else              A[(int64_t)lt * g->n + ls] = x;
        }
}

/* ------------------------------------------------------------------ */
/* Gram matrix G = A^T A (cross-product SVD, Sec. 2.7.1; Eq. 2).        */
/* Each entry is a sequential fma sum over rows l = 0..L-1.             */
/* ------------------------------------------------------------------ */
void or_gram(const double* A, int64_t L, int n, double* G) {
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      double acc = 0.0;
      for (int64_t l = 0; l < L; ++l) acc = fma(A[l * n + i], A[l * n + j], acc);
      G[i * n + j] = acc;
      G[j * n + i] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Symmetric eigensolve of G by Jacobi rotations with round-robin       */
/* (parallel) ordering (Golub & Van Loan, Matrix Computations, 4th ed., */
/* Sec. 8.5).  The right singular vectors of A are the eigenvectors of  */
/* G; the singular values are sqrt(lambda) (Sec. 2.3, Eq. 2-3).         */
/*                                                                      */
/* One sweep = m-1 rounds over the circle-method pairing of m = n       */
/* (rounded up to even) indices.  In a round, each disjoint pair (p,q)  */
/* with |g_pq| > tol gets the classical rotation (c,s,t) computed from  */
/* the matrix at the start of the round; the round applies all row      */
/* rotations, then all column rotations, copies the upper triangle to   */
/* the lower one, and finally sets g_pp, g_qq from the closed form and  */
/* g_pq = 0.  tol = 1e-15 * trace(G).  Sweeps stop after a sweep with   */
/* no rotation, or after 30 sweeps.                                     */
/* Eigenvalues below zero are clamped to zero, sorted descending (stable */
/* for ties), and each eigenvector's largest-magnitude component (lowest */
/* index on ties) is made positive.                                      */
/* ------------------------------------------------------------------ */
static void rr_pair(int round, int i, int m, int* p, int* q) {
  int a, b;
  if (i == 0) { a = m - 1; b = round; }
  else { a = (round + i) % (m - 1); b = (round - i + (m - 1)) % (m - 1); }
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

int or_jacobi(const double* Gin, int n, double* lam, double* Vout) {
  double G[32 * 32], H[32 * 32], G2[32 * 32], V[32 * 32];
  memcpy(G, Gin, sizeof(double) * n * n);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) V[a * n + b] = (a == b) ? 1.0 : 0.0;
  int m = n + (n & 1);
  double tr = 0.0;
  for (int i = 0; i < n; ++i) tr = tr + G[i * n + i];
  double tol = 1e-15 * tr;
  int sweeps = 0;
  for (int sweep = 0; sweep < 30 && n > 1; ++sweep) {
    ++sweeps;
    int rotated = 0;
    for (int round = 0; round < m - 1; ++round) {
      int P[16], Q[16], act[16];
      double c[16], s[16], t[16];
      for (int i = 0; i < m / 2; ++i) {
        rr_pair(round, i, m, &P[i], &Q[i]);
        act[i] = 0;
        if (Q[i] >= n) continue;
        int p = P[i], q = Q[i];
        double apq = G[p * n + q];
        if (!(fabs(apq) > tol)) continue;
        double theta = (G[q * n + q] - G[p * n + p]) / (2.0 * apq);
        double tt;
        if (fabs(theta) > 1e150) tt = 0.5 / theta;
        else tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
        double cc = 1.0 / sqrt(1.0 + tt * tt);
        c[i] = cc; s[i] = tt * cc; t[i] = tt; act[i] = 1;
        ++rotated;
      }
      memcpy(H, G, sizeof(double) * n * n);
      for (int i = 0; i < m / 2; ++i) {
        if (!act[i]) continue;
        int p = P[i], q = Q[i];
        for (int b = 0; b < n; ++b) {
          H[p * n + b] = c[i] * G[p * n + b] - s[i] * G[q * n + b];
          H[q * n + b] = s[i] * G[p * n + b] + c[i] * G[q * n + b];
        }
      }
      memcpy(G2, H, sizeof(double) * n * n);
      for (int i = 0; i < m / 2; ++i) {
        if (!act[i]) continue;
        int p = P[i], q = Q[i];
        for (int a = 0; a < n; ++a) {
          G2[a * n + p] = c[i] * H[a * n + p] - s[i] * H[a * n + q];
          G2[a * n + q] = s[i] * H[a * n + p] + c[i] * H[a * n + q];
        }
      }
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < a; ++b) G2[a * n + b] = G2[b * n + a];
      for (int i = 0; i < m / 2; ++i) {
        if (!act[i]) continue;
        int p = P[i], q = Q[i];
        G2[p * n + p] = G[p * n + p] - t[i] * G[p * n + q];
        G2[q * n + q] = G[q * n + q] + t[i] * G[p * n + q];
        G2[p * n + q] = 0.0;
        G2[q * n + p] = 0.0;
      }
      for (int i = 0; i < m / 2; ++i) {
        if (!act[i]) continue;
        int p = P[i], q = Q[i];
        for (int a = 0; a < n; ++a) {
          double vp = V[a * n + p], vq = V[a * n + q];
          V[a * n + p] = c[i] * vp - s[i] * vq;
          V[a * n + q] = s[i] * vp + c[i] * vq;
        }
      }
      memcpy(G, G2, sizeof(double) * n * n);
    }
    if (rotated == 0) break;
  }
  /* clamp, stable descending order, sign normalisation */
  double d[32];
  int ord[32];
  for (int i = 0; i < n; ++i) { d[i] = G[i * n + i] < 0.0 ? 0.0 : G[i * n + i]; ord[i] = i; }
  for (int i = 1; i < n; ++i) {           /* insertion sort: stable */
    int o = ord[i], j = i - 1;
    while (j >= 0 && d[ord[j]] < d[o]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = o;
  }
  for (int k = 0; k < n; ++k) {
    int src = ord[k];
    lam[k] = d[src];
    int imax = 0;
    double amax = -1.0;
    for (int a = 0; a < n; ++a) {
      double av = fabs(V[a * n + src]);
      if (av > amax) { amax = av; imax = a; }
    }
    double sg = V[imax * n + src] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) Vout[a * n + k] = sg < 0.0 ? -V[a * n + src] : V[a * n + src];
  }
  return sweeps;
}

/* Stored basis: the first r eigenvectors rounded to the field dtype
 * (the basis is stored as plain values, Sec. 2.7.2; its size grows with
 * the patch, Sec. 6).  Vst is n x r row-major. */
void or_round_basis(const double* V, int n, int r, int dtype, double* Vst) {
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < r; ++k) Vst[j * r + k] = to_dt(V[j * n + k], dtype);
}

/* Projection onto the basis, S = C^T P (Sec. 2.5, Eq. 5; Algorithm 1):
 * C[l][k] = sum_j A[l][j] Vst[j][k], sequential fma over j. */
void or_project(const double* A, int64_t L, int n, const double* Vst, int r, double* C) {
  for (int64_t l = 0; l < L; ++l)
    for (int k = 0; k < r; ++k) {
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc = fma(A[l * n + j], Vst[j * r + k], acc);
      C[l * r + k] = acc;
    }
}

/* Uniform coefficient quantizer (stands in for bit-grooming, Sec. 2.5):
 * q = rint(c / delta), ties to even.  Returns 1 if any |c/delta| reaches
 * the code limit (2^24 for f32 fields, 2^30 for f64 fields). */
int or_quantize(const double* C, int64_t cnt, double delta, int dtype, int32_t* q) {
  double lim = dtype == OR_F32 ? OR_QMAX_F32 : OR_QMAX_F64;
  int ovf = 0;
  for (int64_t i = 0; i < cnt; ++i) {
    double y = C[i] / delta;
    if (!(fabs(y) < lim)) { ovf = 1; q[i] = 0; continue; }
    q[i] = (int32_t)nearbyint(y);
  }
  return ovf;
}

/* Dequantized coefficient in the field dtype: dtype(q) * dtype(delta),
 * one rounding in the dtype. */
static double dequant(int32_t q, double delta, int dtype) {
  if (dtype == OR_F32) return (double)((float)q * (float)delta);
  return (double)q * delta;
}

/* Patch reconstruction u = sum_s alpha_s phi_s (Sec. 2.6, Algorithm 2),
 * evaluated in the field dtype as a sequential fma chain over the
 * retained modes k = 0..r-1:  acc = fma(chat[l][k], Vst[j][k], acc).
 * q has leading dimension rq; Vst has leading dimension r... of its own
 * allocation (n x rq).  Output D (L x n) holds dtype values. */
void or_decode(const int32_t* q, int64_t L, int rq, int r, const double* Vst, int n,
               int dtype, double delta, double* D) {
  for (int64_t l = 0; l < L; ++l)
    for (int j = 0; j < n; ++j) {
      if (dtype == OR_F32) {
        float acc = 0.0f;
        for (int k = 0; k < r; ++k)
          acc = fmaf((float)dequant(q[l * rq + k], delta, dtype), (float)Vst[j * rq + k], acc);
        D[l * n + j] = (double)acc;
      } else {
        double acc = 0.0;
        for (int k = 0; k < r; ++k)
          acc = fma(dequant(q[l * rq + k], delta, dtype), Vst[j * rq + k], acc);
        D[l * n + j] = acc;
      }
    }
}

/* Block L2 error e^2 = sum (u - u_hat)^2 (Sec. 2.4), FP64, accumulated in
 * this fixed order: per column j, rows in chunks of 32 (sequential fma
 * inside a chunk), chunk sums added in order, then column sums added in
 * order.  The order is fixed so that any implementation can reproduce it. */
double or_block_err(const double* A, const double* D, int64_t L, int n) {
  double E = 0.0;
  for (int j = 0; j < n; ++j) {
    double sj = 0.0;
    for (int64_t c0 = 0; c0 < L; c0 += 32) {
      int64_t c1 = c0 + 32 < L ? c0 + 32 : L;
      double pc = 0.0;
      for (int64_t l = c0; l < c1; ++l) {
        double d = A[l * n + j] - D[l * n + j];
        pc = fma(d, d, pc);
      }
      sj = sj + pc;
    }
    E = E + sj;
  }
  return E;
}

/* Pointwise correction (the L-infinity guarantee of Sec. 2.4 made
 * explicit): R = x - xhat in FP64, k = rint(R / step) with step = 2 eb;
 * xtilde = xhat if k == 0, else fma(dtype(k), dtype(step), xhat) in the
 * dtype.  A point whose |x - xtilde| > eb (FP64) or |k| > 2^20 becomes an
 * escape (raw value stored, k = 0).  k and esc are in element order
 * e = t_local * M + s_local. */
void or_correct(const double* A, const double* D, int64_t L, int n, int side, int64_t M,
                int dtype, double eb, double step, int32_t* k, uint8_t* esc) {
  for (int64_t l = 0; l < L; ++l)
    for (int j = 0; j < n; ++j) {
      int64_t e = side == 0 ? (int64_t)j * M + l : l * M + j;
      double x = A[l * n + j], xh = D[l * n + j];
      double R = x - xh;
      double y = R / step;
      double kk = nearbyint(y);
      k[e] = 0;
      esc[e] = 0;
      double xt;
      if (kk == 0.0) {
        xt = xh;
      } else if (fabs(kk) > OR_KMAX) {
        esc[e] = 1;
        continue;
      } else {
        if (dtype == OR_F32) xt = (double)fmaf((float)kk, (float)step, (float)xh);
        else xt = fma(kk, step, xh);
      }
      if (fabs(x - xt) > eb) { esc[e] = 1; continue; }
      k[e] = (int32_t)kk;
    }
}

/* ------------------------------------------------------------------ */
/* Bit packing (Sec. 2.7.2: tightly packed DOF arrays).                 */
/* Fields are written LSB-first into little-endian u32 words.           */
/* ------------------------------------------------------------------ */
static uint32_t zz(int32_t v) { return ((uint32_t)v << 1) ^ (uint32_t)(v >> 31); }
static int nbits(uint32_t v) { int b = 0; while (v) { ++b; v >>= 1; } return b; }

static void put_bits(uint32_t* w, uint64_t pos, uint32_t val, int width) {
  if (width == 0) return;
  uint64_t wi = pos >> 5;
  int sh = (int)(pos & 31);
  uint64_t v = (uint64_t)val << sh;
  w[wi] |= (uint32_t)v;
  if (sh + width > 32) w[wi + 1] |= (uint32_t)(v >> 32);
}

static uint32_t get_bits(const uint32_t* w, uint64_t pos, int width) {
  if (width == 0) return 0;
  uint64_t wi = pos >> 5;
  int sh = (int)(pos & 31);
  uint64_t v = w[wi] >> sh;
  if (sh + width > 32) v |= (uint64_t)w[wi + 1] << (32 - sh);
  return (uint32_t)(v & (width == 32 ? 0xffffffffull : ((1ull << width) - 1)));
}

static void wr32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void wr64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static uint32_t rd32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t rd64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

static void put_val(uint8_t* p, double x, int dtype) {
  if (dtype == OR_F32) { float f = (float)x; memcpy(p, &f, 4); }
  else memcpy(p, &x, 8);
}
static double get_val(const uint8_t* p, int dtype) {
  if (dtype == OR_F32) { float f; memcpy(&f, p, 4); return (double)f; }
  double d; memcpy(&d, p, 8); return d;
}

static int64_t raw_record_bytes(int64_t N, int dtype) { return al(16 + N * esize(dtype), 16); }

/* Raw record: header with the RAW flag, then N values in element order. */
static int64_t write_raw(const double* A, int64_t L, int n, int side, int64_t M, int dtype,
                         uint8_t* rec, int64_t cap) {
  int64_t N = L * n;
  int64_t sz = raw_record_bytes(N, dtype);
  if (sz > cap) return OR_ERR_CAPACITY;
  memset(rec, 0, (size_t)sz);
  rec[1] = (uint8_t)(OR_FLAG_RAW | (side ? OR_FLAG_SPATIAL : 0));
  wr32(rec + 12, (uint32_t)sz);
  for (int64_t l = 0; l < L; ++l)
    for (int j = 0; j < n; ++j) {
      int64_t e = side == 0 ? (int64_t)j * M + l : l * M + j;
      put_val(rec + 16 + e * esize(dtype), A[l * n + j], dtype);
    }
  return sz;
}

/* Encoded record:
 *   [0,16)  u8 r, u8 flags, u8 w_k, u8 ib, u32 n_corr, u32 n_esc, u32 nbytes
 *   w_q[r] (u8), padded to 8
 *   Vst: for k < r, for j < n: Vst[j][k] in dtype, padded to 8
 *   q: for k < r: ceil(L*w_q[k]/32) words of zigzag(q[l][k]), l = 0..L-1;
 *      padded to 8
 *   corrections: dense  = ceil(N*w_k/32) words, zigzag(k[e]) for all e;
 *                sparse = ceil(n_corr*(ib+w_k)/32) words, one (ib+w_k)-bit
 *                field per nonzero k in increasing e: e in the low ib bits,
 *                zigzag(k) above; padded to 8
 *   escapes: n_esc u32 element indices (increasing), padded to 8, then
 *            n_esc raw values in dtype, padded to 8
 *   record padded to 16 bytes.
 * Dense is used only when strictly smaller than sparse.
 * With corr_codec = 1 a third form is taken when strictly smaller than both
 * (flag OR_FLAG_RICE): words [0] = number of Rice words, [1] = kr | wv << 8,
 * then ceil(N / OR_RICE_CHUNK) chunk bit offsets, then the Rice words of the
 * corrections with the escaped points as zeros (or_rice_encode). */
int64_t or_pack_record(int r, int side, int n, int64_t L, int64_t M, int dtype,
                       const double* Vst, const int32_t* q, const int32_t* k,
                       const uint8_t* esc, const double* A, uint8_t* rec, int64_t cap, int corr_codec) {
  int64_t N = L * n;
  int es = esize(dtype);
  uint8_t wq[32];
  for (int c = 0; c < r; ++c) {
    uint32_t mx = 0;
    for (int64_t l = 0; l < L; ++l) { uint32_t z = zz(q[l * r + c]); if (z > mx) mx = z; }
    wq[c] = (uint8_t)nbits(mx);
  }
  uint32_t kmx = 0;
  int64_t ncorr = 0, nesc = 0;
  for (int64_t e = 0; e < N; ++e) {
    if (esc[e]) { ++nesc; continue; }
    if (k[e] != 0) { ++ncorr; uint32_t z = zz(k[e]); if (z > kmx) kmx = z; }
  }
  int wk = nbits(kmx);
  int ib = nbits((uint32_t)(N - 1));
  int64_t dense_w = (N * wk + 31) / 32, sparse_w = (ncorr * (ib + wk) + 31) / 32;
  int dense = (wk > 0) && (dense_w < sparse_w);
  int64_t corr_w = wk == 0 ? 0 : (dense ? dense_w : sparse_w);
  int rice = 0, kr = 0, wv = 0;
  int32_t* kz = NULL;
  int64_t nchunks = (N + OR_RICE_CHUNK - 1) / OR_RICE_CHUNK, rice_words = 0;
  if (corr_codec == 1 && wk > 0) {
    kz = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    for (int64_t e = 0; e < N; ++e) kz[e] = esc[e] ? 0 : k[e];
    or_rice_choose(kz, N, OR_RICE_CHUNK, &kr, &wv);
    rice_words = (or_rice_bits(kz, N, OR_RICE_CHUNK, kr, wv) + 31) / 32;
    if (2 + nchunks + rice_words < corr_w) {
      rice = 1;
      dense = 0;
      corr_w = 2 + nchunks + rice_words;
    }
  }

  int64_t off_wq = 16;
  int64_t off_v = off_wq + al(r, 8);
  int64_t off_q = off_v + al((int64_t)n * r * es, 8);
  int64_t qwords = 0;
  for (int c = 0; c < r; ++c) qwords += (L * wq[c] + 31) / 32;
  int64_t off_c = off_q + al(qwords * 4, 8);
  int64_t off_ei = off_c + al(corr_w * 4, 8);
  int64_t off_ev = off_ei + al(nesc * 4, 8);
  int64_t sz = al(off_ev + al(nesc * es, 8), 16);
  if (sz > cap) { free(kz); return OR_ERR_CAPACITY; }
  memset(rec, 0, (size_t)sz);
  rec[0] = (uint8_t)r;
  rec[1] = (uint8_t)((side ? OR_FLAG_SPATIAL : 0) | (dense ? OR_FLAG_DENSE : 0) | (rice ? OR_FLAG_RICE : 0));
  rec[2] = (uint8_t)wk;
  rec[3] = (uint8_t)ib;
  wr32(rec + 4, (uint32_t)ncorr);
  wr32(rec + 8, (uint32_t)nesc);
  wr32(rec + 12, (uint32_t)sz);
  for (int c = 0; c < r; ++c) rec[off_wq + c] = wq[c];
  for (int c = 0; c < r; ++c)
    for (int j = 0; j < n; ++j) put_val(rec + off_v + ((int64_t)c * n + j) * es, Vst[j * r + c], dtype);
  uint32_t* qw = (uint32_t*)(rec + off_q);
  int64_t wbase = 0;
  for (int c = 0; c < r; ++c) {
    for (int64_t l = 0; l < L; ++l) put_bits(qw + wbase, (uint64_t)l * wq[c], zz(q[l * r + c]), wq[c]);
    wbase += (L * wq[c] + 31) / 32;
  }
  uint32_t* cw = (uint32_t*)(rec + off_c);
  if (rice) {
    cw[0] = (uint32_t)rice_words;
    cw[1] = (uint32_t)kr | ((uint32_t)wv << 8);
    or_rice_encode(kz, N, OR_RICE_CHUNK, kr, wv, cw + 2 + nchunks, rice_words, cw + 2);
  } else if (wk > 0) {
    if (dense) {
      for (int64_t e = 0; e < N; ++e) put_bits(cw, (uint64_t)e * wk, esc[e] ? 0u : zz(k[e]), wk);
    } else {
      int64_t i = 0;
      for (int64_t e = 0; e < N; ++e) {
        if (esc[e] || k[e] == 0) continue;
        uint64_t pos = (uint64_t)i * (ib + wk);
        put_bits(cw, pos, (uint32_t)e, ib);
        put_bits(cw, pos + ib, zz(k[e]), wk);
        ++i;
      }
    }
  }
  int64_t i = 0;
  for (int64_t e = 0; e < N; ++e) {
    if (!esc[e]) continue;
    wr32(rec + off_ei + i * 4, (uint32_t)e);
    int64_t l = side == 0 ? e % M : e / M;
    int j = side == 0 ? (int)(e / M) : (int)(e % M);
    put_val(rec + off_ev + i * es, A[l * n + j], dtype);
    ++i;
  }
  free(kz);
  return sz;
}

int64_t or_max_record_bytes(const or_params* p, int64_t b) {
  or_geom g;
  or_block_geom(p, b, &g);
  return raw_record_bytes(g.N, p->dtype);
}

/* ------------------------------------------------------------------ */
/* One block, Algorithm 1 step 3 (per patch):                           */
/*   project -> quantize -> smallest prefix meeting eps_l by bisection   */
/*   -> (pointwise modes) correction -> pack (raw if not smaller).       */
/* ------------------------------------------------------------------ */
int64_t or_block_compress(const or_params* p, const void* field, int64_t b, const or_var* vars,
                          uint8_t* rec, int64_t rec_cap, or_trace* tr,
                          double* G_out, double* lam_out, double* V_out, double* Vst_out,
                          int32_t* q_out, int32_t* k_out, int want_linear) {
  or_geom g;
  or_block_geom(p, b, &g);
  const or_var* o = &vars[g.v];
  int n = g.n;
  int64_t L = g.L, N = g.N;
  int rcap = p->rank_cap < n ? p->rank_cap : n;
  double* A = (double*)malloc(sizeof(double) * N);
  double* D = (double*)malloc(sizeof(double) * N);
  double* C = (double*)malloc(sizeof(double) * (L * (rcap > 0 ? rcap : 1)));
  int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (L * (rcap > 0 ? rcap : 1)));
  int32_t* kk = (int32_t*)calloc((size_t)N, sizeof(int32_t));
  uint8_t* esc = (uint8_t*)calloc((size_t)N, 1);
  double G[32 * 32], lam[32], V[32 * 32], Vst[32 * 32];
  or_gather(p, field, &g, A);
  or_gram(A, L, n, G);
  if (G_out) memcpy(G_out, G, sizeof(double) * n * n);
  int sweeps = 0;
  if (p->basis && p->basis_n == n) {
    /* the given modes, as given; lam_k = v_k^T G v_k, the energy of mode k */
    memcpy(V, p->basis, sizeof(double) * n * n);
    for (int k = 0; k < n; ++k) {
      double e = 0.0;
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) e += V[a * n + k] * G[a * n + c] * V[c * n + k];
      lam[k] = e;
    }
  } else {
    sweeps = or_jacobi(G, n, lam, V);
  }
  or_round_basis(V, n, rcap, p->dtype, Vst);
  if (lam_out) memcpy(lam_out, lam, sizeof(double) * n);
  if (V_out) memcpy(V_out, V, sizeof(double) * n * n);
  if (Vst_out) memcpy(Vst_out, Vst, sizeof(double) * n * rcap);
  or_project(A, L, n, Vst, rcap, C);
  int ovf = or_quantize(C, L * rcap, o->delta, p->dtype, q);
  if (q_out) memcpy(q_out, q, sizeof(int32_t) * L * rcap);
  double el2 = el2_of(p, o, N);
  if (tr) {
    memset(tr, 0, sizeof(*tr));
    for (int i = 0; i < 33; ++i) tr->E[i] = NAN;
    tr->n = n; tr->side = g.side; tr->rcap = rcap; tr->L = L; tr->N = N;
    tr->sweeps = sweeps; tr->el2 = el2; tr->overflow = ovf; tr->lin_r = -1;
  }
  int64_t sz;
  int raw = ovf;
  int r = 0;
  if (!raw) {
    /* bisection over r in [0, rcap]: pass(r) <=> E(r) <= eps_l^2 */
    int lo = 0, hi = rcap, np = 0;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      or_decode(q, L, rcap, mid, Vst, n, p->dtype, o->delta, D);
      double E = or_block_err(A, D, L, n);
      if (tr) { tr->E[mid] = E; if (np < 8) tr->probe_r[np] = mid; }
      ++np;
      if (E <= el2) hi = mid; else lo = mid + 1;
    }
    r = lo;
    if (tr) tr->nprobes = np;
    or_decode(q, L, rcap, r, Vst, n, p->dtype, o->delta, D);
    if (p->eb_type == OR_EB_NRMSE) {
      double E = or_block_err(A, D, L, n);
      if (tr && isnan(tr->E[r])) tr->E[r] = E;
      if (!(E <= el2)) raw = 1;    /* keep the L2 budget: store this block raw */
    } else {
      or_correct(A, D, L, n, g.side, g.M, p->dtype, o->eb, o->step, kk, esc);
    }
    if (tr && want_linear) {
      int lr = -1;
      for (int rr = 0; rr <= rcap && lr < 0; ++rr) {
        or_decode(q, L, rcap, rr, Vst, n, p->dtype, o->delta, D);
        if (or_block_err(A, D, L, n) <= el2) lr = rr;
      }
      tr->lin_r = lr < 0 ? rcap : lr;
    }
  }
  if (!raw) {
    /* q for the record: first r columns, leading dimension r */
    int32_t* qr = (int32_t*)malloc(sizeof(int32_t) * (L * (r > 0 ? r : 1)));
    double Vr[32 * 32];
    for (int64_t l = 0; l < L; ++l)
      for (int c = 0; c < r; ++c) qr[l * r + c] = q[l * rcap + c];
    for (int j = 0; j < n; ++j)
      for (int c = 0; c < r; ++c) Vr[j * r + c] = Vst[j * rcap + c];
    int64_t rawsz = raw_record_bytes(N, p->dtype);
    uint8_t* tmp = (uint8_t*)malloc((size_t)(rawsz + 4096 + 64 * (int64_t)n * n));
    sz = or_pack_record(r, g.side, n, L, g.M, p->dtype, Vr, qr, kk, esc, A, tmp,
                        rawsz + 4096 + 64 * (int64_t)n * n, p->corr_codec);
    if (sz >= rawsz) {
      raw = 1;
    } else if (sz > rec_cap) {
      sz = OR_ERR_CAPACITY;
    } else {
      memcpy(rec, tmp, (size_t)sz);
    }
    free(tmp);
    free(qr);
    if (tr && !raw) {
      tr->r = r;
      tr->n_corr = rd32(rec + 4);
      tr->n_esc = rd32(rec + 8);
      tr->wk = rec[2]; tr->ib = rec[3]; tr->dense = (rec[1] & OR_FLAG_DENSE) ? 1 : 0;
    }
  }
  if (raw) {
    sz = write_raw(A, L, n, g.side, g.M, p->dtype, rec, rec_cap);
    if (tr) { tr->raw = 1; tr->r = 0; }
  }
  if (k_out) memcpy(k_out, kk, sizeof(int32_t) * N);
  if (tr) tr->nbytes = sz;
  free(A); free(D); free(C); free(q); free(kk); free(esc);
  return sz;
}

/* ------------------------------------------------------------------ */
/* Whole field (Algorithm 1 step 3 over all patches; Sec. 2.7.2 layout: */
/* addressable header, offsets from an exclusive scan of record sizes,  */
/* then the packed records).                                            */
/* ------------------------------------------------------------------ */
static int64_t nblk_range(const or_params* p, int64_t* b0) {
  int64_t nb = or_num_blocks(p);
  int64_t e = p->block_end < 0 ? nb : p->block_end;
  *b0 = p->block_begin;
  return e - p->block_begin;
}

int64_t or_compress_bound(const or_params* p) {
  if (or_validate(p) != OR_OK) return -1;
  int64_t b0, nb = nblk_range(p, &b0);
  int64_t offp = al(OR_HDR + (int64_t)OR_VARREC * p->nvars, 16);
  int64_t pay = al(offp + 8 * (nb + 1), 16);
  int64_t tot = pay;
  for (int64_t b = 0; b < nb; ++b) tot += or_max_record_bytes(p, b0 + b);
  return tot;
}

int or_compress(const or_params* p, const void* field, void* out, int64_t cap,
                int64_t* out_bytes, or_trace* traces, int nthreads) {
  int st = or_validate(p);
  if (st != OR_OK) return st;
  or_var vars[64];
  if (p->nvars > 64) return OR_ERR_INVALID_ARG;
  st = or_resolve(p, field, vars);
  if (st != OR_OK) return st;
  int64_t b0, nb = nblk_range(p, &b0);
  int64_t* sizes = (int64_t*)calloc((size_t)(nb + 1), sizeof(int64_t));
  uint8_t** recs = (uint8_t**)calloc((size_t)(nb > 0 ? nb : 1), sizeof(uint8_t*));
  int err = OR_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < nb; ++i) {
    int64_t cap_b = or_max_record_bytes(p, b0 + i);
    recs[i] = (uint8_t*)malloc((size_t)cap_b);
    int64_t s = or_block_compress(p, field, b0 + i, vars, recs[i], cap_b,
                                  traces ? &traces[i] : NULL, NULL, NULL, NULL, NULL, NULL, NULL, 0);
    if (s < 0) err = (int)s;
    sizes[i] = s < 0 ? 0 : s;
  }
  if (err != OR_OK) {
    for (int64_t i = 0; i < nb; ++i) free(recs[i]);
    free(recs); free(sizes);
    return err;
  }
  int64_t offp = al(OR_HDR + (int64_t)OR_VARREC * p->nvars, 16);
  int64_t payp = al(offp + 8 * (nb + 1), 16);
  int64_t acc = 0;
  int64_t* offs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
  for (int64_t i = 0; i < nb; ++i) { offs[i] = acc; acc += sizes[i]; }   /* exclusive scan */
  offs[nb] = acc;
  int64_t total = payp + acc;
  if (out_bytes) *out_bytes = total;
  if (!out || total > cap) {
    for (int64_t i = 0; i < nb; ++i) free(recs[i]);
    free(recs); free(sizes); free(offs);
    return out ? OR_ERR_CAPACITY : OR_OK;
  }
  uint8_t* o = (uint8_t*)out;
  memset(o, 0, (size_t)payp);
  wr32(o + 0, OR_MAGIC);
  wr32(o + 4, OR_VERSION);
  wr32(o + 8, OR_HDR);
  wr32(o + 12, (uint32_t)p->nvars);
  for (int a = 0; a < 4; ++a) wr64(o + 16 + 8 * a, (uint64_t)p->dims[a]);
  for (int a = 0; a < 4; ++a) wr32(o + 48 + 4 * a, (uint32_t)p->block[a]);
  o[64] = (uint8_t)p->dtype;
  o[65] = (uint8_t)p->eb_type;
  o[66] = 0;   /* precision: FP64 */
  o[67] = 0;   /* rank mode: search */
  wr32(o + 68, (uint32_t)p->rank_cap);
  wr64(o + 72, (uint64_t)b0);
  wr64(o + 80, (uint64_t)(b0 + nb));
  wr64(o + 88, (uint64_t)or_num_blocks(p));
  wr64(o + 96, (uint64_t)OR_HDR);
  wr64(o + 104, (uint64_t)offp);
  wr64(o + 112, (uint64_t)payp);
  wr64(o + 120, (uint64_t)total);
  for (int v = 0; v < p->nvars; ++v) {
    uint8_t* vr = o + OR_HDR + OR_VARREC * v;
    memcpy(vr + 0, &vars[v].eb_user, 8);
    memcpy(vr + 8, &vars[v].eb, 8);
    memcpy(vr + 16, &vars[v].delta, 8);
    memcpy(vr + 24, &vars[v].step, 8);
  }
  for (int64_t i = 0; i <= nb; ++i) wr64(o + offp + 8 * i, (uint64_t)offs[i]);
  for (int64_t i = 0; i < nb; ++i) {
    memcpy(o + payp + offs[i], recs[i], (size_t)sizes[i]);
    free(recs[i]);
  }
  free(recs); free(sizes); free(offs);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Decompression (Sec. 2.6, Algorithm 2): per record, unpack, decode     */
/* per the fma-chain contract, add corrections, overwrite escapes, and   */
/* assemble the block into the field.                                   */
/* ------------------------------------------------------------------ */
int or_decompress(const void* stream, int64_t bytes, void* out, int64_t out_cap, int nthreads) {
  const uint8_t* s = (const uint8_t*)stream;
  if (bytes < OR_HDR || rd32(s) != OR_MAGIC || rd32(s + 4) != OR_VERSION) return OR_ERR_CORRUPT;
  or_params p;
  memset(&p, 0, sizeof(p));
  p.nvars = (int32_t)rd32(s + 12);
  if (p.nvars < 1 || p.nvars > 64) return OR_ERR_CORRUPT;
  for (int a = 0; a < 4; ++a) p.dims[a] = (int64_t)rd64(s + 16 + 8 * a);
  for (int a = 0; a < 4; ++a) p.block[a] = (int32_t)rd32(s + 48 + 4 * a);
  p.dtype = s[64];
  p.eb_type = s[65];
  p.rank_cap = (int32_t)rd32(s + 68);
  p.block_begin = (int64_t)rd64(s + 72);
  p.block_end = (int64_t)rd64(s + 80);
  double ebs[64];
  int64_t offp = (int64_t)rd64(s + 104), payp = (int64_t)rd64(s + 112), total = (int64_t)rd64(s + 120);
  if ((int64_t)(OR_HDR + OR_VARREC * p.nvars) > bytes) return OR_ERR_CORRUPT;
  for (int v = 0; v < p.nvars; ++v) memcpy(&ebs[v], s + OR_HDR + OR_VARREC * v, 8);
  p.eb = ebs;
  if (or_validate(&p) != OR_OK) return OR_ERR_CORRUPT;
  if ((int64_t)rd64(s + 88) != or_num_blocks(&p)) return OR_ERR_CORRUPT;
  int64_t nb = p.block_end - p.block_begin;
  if (total != bytes || offp != al(OR_HDR + (int64_t)OR_VARREC * p.nvars, 16) ||
      payp != al(offp + 8 * (nb + 1), 16) || payp > bytes) return OR_ERR_CORRUPT;
  int64_t K = p.dims[0] * p.dims[1] * p.dims[2] * p.dims[3];
  int es = esize(p.dtype);
  if (out_cap < K * p.nvars * es) return OR_ERR_CAPACITY;
  int err = OR_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t i = 0; i < nb; ++i) {
    int64_t o0 = (int64_t)rd64(s + offp + 8 * i), o1 = (int64_t)rd64(s + offp + 8 * (i + 1));
    if (o0 < 0 || o1 < o0 || payp + o1 > bytes) { err = OR_ERR_CORRUPT; continue; }
    const uint8_t* rec = s + payp + o0;
    or_geom g;
    or_block_geom(&p, p.block_begin + i, &g);
    const uint8_t* vr = s + OR_HDR + OR_VARREC * g.v;
    double delta, step;
    memcpy(&delta, vr + 16, 8);
    memcpy(&step, vr + 24, 8);
    int64_t L = g.L, N = g.N, M = g.M;
    int n = g.n;
    int r = rec[0], flags = rec[1], wk = rec[2], ib = rec[3];
    int64_t ncorr = rd32(rec + 4), nesc = rd32(rec + 8), nbytes = rd32(rec + 12);
    if (nbytes != o1 - o0 || nbytes < 16) { err = OR_ERR_CORRUPT; continue; }
    double* X = (double*)malloc(sizeof(double) * N);    /* element order */
    if (flags & OR_FLAG_RAW) {
      if (16 + N * es > nbytes) { err = OR_ERR_CORRUPT; free(X); continue; }
      for (int64_t e = 0; e < N; ++e) X[e] = get_val(rec + 16 + e * es, p.dtype);
    } else {
      int rcap = p.rank_cap < n ? p.rank_cap : n;
      if (r > rcap || wk > 32 || ib != nbits((uint32_t)(N - 1)) || ncorr > N || nesc > N ||
          ((flags & OR_FLAG_SPATIAL) ? 1 : 0) != g.side) {
        err = OR_ERR_CORRUPT; free(X); continue;
      }
      const uint8_t* wq = rec + 16;
      int64_t off_v = 16 + al(r, 8);
      int64_t off_q = off_v + al((int64_t)n * r * es, 8);
      int64_t qwords = 0;
      int bad = 0;
      for (int c = 0; c < r; ++c) { if (wq[c] > 32) bad = 1; qwords += (L * wq[c] + 31) / 32; }
      int dense = (flags & OR_FLAG_DENSE) ? 1 : 0;
      int rice = (flags & OR_FLAG_RICE) ? 1 : 0;
      int64_t off_c = off_q + al(qwords * 4, 8);
      int64_t nchunks = (N + OR_RICE_CHUNK - 1) / OR_RICE_CHUNK, rice_words = 0;
      if (rice && (wk == 0 || dense || off_c + 8 > nbytes)) { err = OR_ERR_CORRUPT; free(X); continue; }
      if (rice) rice_words = rd32(rec + off_c);
      int64_t corr_w = wk == 0 ? 0
                       : rice ? 2 + nchunks + rice_words
                              : (dense ? (N * wk + 31) / 32 : (ncorr * (ib + wk) + 31) / 32);
      int64_t off_ei = off_c + al(corr_w * 4, 8);
      int64_t off_ev = off_ei + al(nesc * 4, 8);
      int64_t need = al(off_ev + al(nesc * es, 8), 16);
      if (bad || need != nbytes) { err = OR_ERR_CORRUPT; free(X); continue; }
      double Vst[32 * 32];
      for (int c = 0; c < r; ++c)
        for (int j = 0; j < n; ++j) Vst[j * r + c] = get_val(rec + off_v + ((int64_t)c * n + j) * es, p.dtype);
      int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (L * (r > 0 ? r : 1)));
      const uint32_t* qw = (const uint32_t*)(rec + off_q);
      int64_t wbase = 0;
      for (int c = 0; c < r; ++c) {
        for (int64_t l = 0; l < L; ++l) {
          uint32_t z = get_bits(qw + wbase, (uint64_t)l * wq[c], wq[c]);
          q[l * r + c] = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
        }
        wbase += (L * wq[c] + 31) / 32;
      }
      double* D = (double*)malloc(sizeof(double) * N);
      or_decode(q, L, r, r, Vst, n, p.dtype, delta, D);
      for (int64_t l = 0; l < L; ++l)
        for (int j = 0; j < n; ++j) {
          int64_t e = g.side == 0 ? (int64_t)j * M + l : l * M + j;
          X[e] = D[l * n + j];
        }
      const uint32_t* cw = (const uint32_t*)(rec + off_c);
      if (rice) {
        const int kr = (int)(cw[1] & 0xffu), wv = (int)((cw[1] >> 8) & 0xffu);
        int32_t* kd = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
        if (kr > 20 || wv > 32 ||
            or_rice_decode(cw + 2 + nchunks, rice_words, cw + 2, N, OR_RICE_CHUNK, kr, wv, kd) != 0) {
          bad = 1;
        } else {
          for (int64_t e = 0; e < N; ++e) {
            const int32_t kv = kd[e];
            if (kv == 0) continue;
            if (p.dtype == OR_F32) X[e] = (double)fmaf((float)kv, (float)step, (float)X[e]);
            else X[e] = fma((double)kv, step, X[e]);
          }
        }
        free(kd);
      } else if (wk > 0) {
        if (dense) {
          for (int64_t e = 0; e < N; ++e) {
            uint32_t z = get_bits(cw, (uint64_t)e * wk, wk);
            int32_t kv = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
            if (kv != 0) {
              if (p.dtype == OR_F32) X[e] = (double)fmaf((float)kv, (float)step, (float)X[e]);
              else X[e] = fma((double)kv, step, X[e]);
            }
          }
        } else {
          for (int64_t ci = 0; ci < ncorr; ++ci) {
            uint64_t pos = (uint64_t)ci * (ib + wk);
            int64_t e = get_bits(cw, pos, ib);
            uint32_t z = get_bits(cw, pos + ib, wk);
            int32_t kv = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
            if (e >= N) { bad = 1; break; }
            if (p.dtype == OR_F32) X[e] = (double)fmaf((float)kv, (float)step, (float)X[e]);
            else X[e] = fma((double)kv, step, X[e]);
          }
        }
      }
      for (int64_t ei = 0; ei < nesc; ++ei) {
        int64_t e = rd32(rec + off_ei + 4 * ei);
        if (e >= N) { bad = 1; break; }
        X[e] = get_val(rec + off_ev + ei * es, p.dtype);
      }
      free(q); free(D);
      if (bad) { err = OR_ERR_CORRUPT; free(X); continue; }
    }
    /* assemble (Algorithm 2: union of patches) */
    int64_t nx = p.dims[0], ny = p.dims[1], P = nx * ny * p.dims[2];
    int64_t base = (int64_t)g.v * K;
    for (int32_t lt = 0; lt < g.st; ++lt)
      for (int32_t lz = 0; lz < g.sz; ++lz)
        for (int32_t ly = 0; ly < g.sy; ++ly)
          for (int32_t lx = 0; lx < g.sx; ++lx) {
            int64_t ls = ((int64_t)lz * g.sy + ly) * g.sx + lx;
            int64_t gi = base + (g.t0 + lt) * P + (g.z0 + lz) * nx * ny + (g.y0 + ly) * nx + (g.x0 + lx);
            double x = X[(int64_t)lt * M + ls];
            if (p.dtype == OR_F32) ((float*)out)[gi] = (float)x;
            else ((double*)out)[gi] = x;
          }
    free(X);
  }
  return err;
}

/* ------------------------------------------------------------------ */
/* Rice-coded corrections: a record section that or_pack_record takes  */
/* with corr_codec = 1 (flag 8) where it is smaller (the lossless      */
/* stage of the stream format).  The corrections k[0..N) of a block,   */
/* in element order,                                                    */
/* are cut into chunks of `chunk` elements.  Within a chunk every       */
/* nonzero is written as the Rice code of the zeros before it (counted  */
/* from the chunk start or the previous nonzero), then zigzag(k) - 1 in */
/* wv bits; one more Rice code gives the zeros up to the chunk end.  The */
/* Rice code of r with parameter kr: (r >> kr) one bits, a zero bit, the */
/* kr low bits of r.  Bits are LSB-first in 32-bit words; chunk c starts */
/* at bit off[c], the chunks one after another from bit 0, so that the  */
/* chunks decode independently.                                         */
/* ------------------------------------------------------------------ */
static uint32_t rz_zig(int32_t v) { return ((uint32_t)v << 1) ^ (uint32_t)(v >> 31); }
static int32_t rz_unzig(uint32_t u) { return (int32_t)(u >> 1) ^ -(int32_t)(u & 1u); }
static int rz_width(uint32_t x) { int w = 0; while (x) { ++w; x >>= 1; } return w; }

int64_t or_rice_bits(const int32_t* k, int64_t N, int chunk, int kr, int wv) {
  int64_t bits = 0;
  for (int64_t c0 = 0; c0 < N; c0 += chunk) {
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    int64_t run = 0;
    for (int64_t e = c0; e < c1; ++e) {
      if (k[e] == 0) { ++run; continue; }
      bits += (run >> kr) + 1 + kr + wv;
      run = 0;
    }
    bits += (run >> kr) + 1 + kr;
  }
  return bits;
}

/* wv: the bit width of the largest zigzag(k) - 1 over the nonzeros; kr in
 * [0, 20] with the fewest bits (the smallest such kr). */
void or_rice_choose(const int32_t* k, int64_t N, int chunk, int* kr_out, int* wv_out) {
  uint32_t mx = 0;
  for (int64_t e = 0; e < N; ++e)
    if (k[e] != 0 && rz_zig(k[e]) - 1u > mx) mx = rz_zig(k[e]) - 1u;
  const int wv = rz_width(mx);
  int best = 0;
  int64_t bb = -1;
  for (int kr = 0; kr <= 20; ++kr) {
    const int64_t b = or_rice_bits(k, N, chunk, kr, wv);
    if (bb < 0 || b < bb) { bb = b; best = kr; }
  }
  *kr_out = best;
  *wv_out = wv;
}

static int rz_put(uint32_t* w, int64_t cap_words, int64_t pos, uint32_t v, int width) {
  for (int i = 0; i < width; ++i) {
    const int64_t p = pos + i;
    if ((p >> 5) >= cap_words) return -1;
    if ((v >> i) & 1u) w[p >> 5] |= 1u << (p & 31);
  }
  return 0;
}

static int rz_code(uint32_t* w, int64_t cap, int64_t* pos, int64_t run, int kr) {
  for (int64_t i = 0; i < (run >> kr); ++i) {
    if (rz_put(w, cap, *pos, 1u, 1) < 0) return -1;
    ++*pos;
  }
  if (rz_put(w, cap, *pos, 0u, 1) < 0) return -1;
  ++*pos;
  if (rz_put(w, cap, *pos, (uint32_t)(run & ((1ll << kr) - 1)), kr) < 0) return -1;
  *pos += kr;
  return 0;
}

/* Returns the bits written (-1 if cap_words is too small); off gets the bit
 * offset of each of the ceil(N / chunk) chunks. */
int64_t or_rice_encode(const int32_t* k, int64_t N, int chunk, int kr, int wv, uint32_t* words,
                       int64_t cap_words, uint32_t* off) {
  memset(words, 0, sizeof(uint32_t) * (size_t)cap_words);
  int64_t pos = 0, c = 0;
  for (int64_t c0 = 0; c0 < N; c0 += chunk, ++c) {
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    off[c] = (uint32_t)pos;
    int64_t run = 0;
    for (int64_t e = c0; e < c1; ++e) {
      if (k[e] == 0) { ++run; continue; }
      if (rz_code(words, cap_words, &pos, run, kr) < 0) return -1;
      if (rz_put(words, cap_words, pos, rz_zig(k[e]) - 1u, wv) < 0) return -1;
      pos += wv;
      run = 0;
    }
    if (rz_code(words, cap_words, &pos, run, kr) < 0) return -1;
  }
  return pos;
}

static int rz_get(const uint32_t* w, int64_t nwords, int64_t pos, int width, uint32_t* v) {
  uint32_t x = 0;
  for (int i = 0; i < width; ++i) {
    const int64_t p = pos + i;
    if ((p >> 5) >= nwords) return -1;
    x |= ((w[p >> 5] >> (p & 31)) & 1u) << i;
  }
  *v = x;
  return 0;
}

/* 0, or -1 for a malformed section (a run past its chunk, a read past the
 * words). */
int or_rice_decode(const uint32_t* words, int64_t nwords, const uint32_t* off, int64_t N, int chunk, int kr,
                   int wv, int32_t* k) {
  int64_t c = 0;
  for (int64_t c0 = 0; c0 < N; c0 += chunk, ++c) {
    const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
    int64_t pos = off[c], e = c0;
    for (;;) {
      int64_t q = 0;
      uint32_t bit = 1;
      while (1) {
        if (rz_get(words, nwords, pos, 1, &bit) < 0) return -1;
        ++pos;
        if (!bit) break;
        if (((q + 1) << kr) > c1 - e) return -1;
        ++q;
      }
      uint32_t lo = 0;
      if (rz_get(words, nwords, pos, kr, &lo) < 0) return -1;
      pos += kr;
      const int64_t run = (q << kr) | lo;
      if (run > c1 - e) return -1;
      for (int64_t i = 0; i < run; ++i) k[e + i] = 0;
      e += run;
      if (e == c1) break;
      uint32_t v = 0;
      if (rz_get(words, nwords, pos, wv, &v) < 0) return -1;
      pos += wv;
      k[e++] = rz_unzig(v + 1u);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Record parser: the inverse of or_pack_record (Sec. 2.7.2 record      */
/* layout), for tests that replay a stored record through the steps     */
/* above.  Given the block's geometry it returns the rank, the flags,   */
/* the stored modes Vst (n x r, leading dimension r), the coefficient   */
/* codes q (L x r, leading dimension r), the corrections k and the      */
/* escape marks esc (element order), and the raw escaped values escval  */
/* (element order, 0 elsewhere).  Raw records give r = 0, flags with    */
/* OR_FLAG_RAW and the values in escval.  0, or OR_ERR_CORRUPT when the */
/* record does not follow the layout exactly.                           */
/* ------------------------------------------------------------------ */
int or_parse_record(const uint8_t* rec, int64_t nbytes, int side, int n, int64_t L, int64_t M, int dtype,
                    int* r_out, int* flags_out, double* Vst, int32_t* q, int32_t* k, uint8_t* esc,
                    double* escval) {
  const int64_t N = L * n;
  const int es = esize(dtype);
  if (nbytes < 16 || (int64_t)rd32(rec + 12) != nbytes) return OR_ERR_CORRUPT;
  const int r = rec[0], flags = rec[1], wk = rec[2], ib = rec[3];
  const int64_t ncorr = rd32(rec + 4), nesc = rd32(rec + 8);
  *r_out = 0;
  *flags_out = flags;
  memset(k, 0, sizeof(int32_t) * (size_t)N);
  memset(esc, 0, (size_t)N);
  memset(escval, 0, sizeof(double) * (size_t)N);
  if (((flags & OR_FLAG_SPATIAL) ? 1 : 0) != side) return OR_ERR_CORRUPT;
  if (flags & OR_FLAG_RAW) {
    if (nbytes != raw_record_bytes(N, dtype)) return OR_ERR_CORRUPT;
    for (int64_t e = 0; e < N; ++e) escval[e] = get_val(rec + 16 + e * es, dtype);
    return OR_OK;
  }
  if ((flags & ~(OR_FLAG_SPATIAL | OR_FLAG_DENSE | OR_FLAG_RICE)) != 0) return OR_ERR_CORRUPT;
  const int rice = (flags & OR_FLAG_RICE) ? 1 : 0;
  if (rice && (wk == 0 || (flags & OR_FLAG_DENSE))) return OR_ERR_CORRUPT;
  if (r > n || wk > 32 || ib != nbits((uint32_t)(N - 1)) || ncorr > N || nesc > N) return OR_ERR_CORRUPT;
  const uint8_t* wq = rec + 16;
  const int64_t off_v = 16 + al(r, 8);
  const int64_t off_q = off_v + al((int64_t)n * r * es, 8);
  int64_t qwords = 0;
  for (int c = 0; c < r; ++c) {
    if (wq[c] > 32) return OR_ERR_CORRUPT;
    qwords += (L * wq[c] + 31) / 32;
  }
  const int dense = (flags & OR_FLAG_DENSE) ? 1 : 0;
  const int64_t off_c = off_q + al(qwords * 4, 8);
  const int64_t nchunks = (N + OR_RICE_CHUNK - 1) / OR_RICE_CHUNK;
  int64_t rice_words = 0;
  if (rice) {
    if (off_c + 8 > nbytes) return OR_ERR_CORRUPT;
    rice_words = rd32(rec + off_c);
  }
  const int64_t corr_w = wk == 0 ? 0
                         : rice ? 2 + nchunks + rice_words
                                : (dense ? (N * wk + 31) / 32 : (ncorr * (ib + wk) + 31) / 32);
  const int64_t off_ei = off_c + al(corr_w * 4, 8);
  const int64_t off_ev = off_ei + al(nesc * 4, 8);
  if (al(off_ev + al(nesc * es, 8), 16) != nbytes) return OR_ERR_CORRUPT;
  for (int c = 0; c < r; ++c)
    for (int j = 0; j < n; ++j) Vst[j * r + c] = get_val(rec + off_v + ((int64_t)c * n + j) * es, dtype);
  const uint32_t* qw = (const uint32_t*)(rec + off_q);
  int64_t wbase = 0;
  for (int c = 0; c < r; ++c) {
    for (int64_t l = 0; l < L; ++l) {
      const uint32_t z = get_bits(qw + wbase, (uint64_t)l * wq[c], wq[c]);
      q[l * r + c] = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
    }
    wbase += (L * wq[c] + 31) / 32;
  }
  const uint32_t* cw = (const uint32_t*)(rec + off_c);
  if (rice) {
    /* the Rice section: its decoder, then the counts the header claims */
    const int kr = (int)(cw[1] & 0xFFu), wv = (int)((cw[1] >> 8) & 0xFFu);
    if ((cw[1] >> 16) != 0 || kr > 20 || wv > 32) return OR_ERR_CORRUPT;
    if (or_rice_decode(cw + 2 + nchunks, rice_words, cw + 2, N, OR_RICE_CHUNK, kr, wv, k) != 0)
      return OR_ERR_CORRUPT;
    int64_t nz = 0;
    uint32_t kmx = 0;
    for (int64_t e = 0; e < N; ++e)
      if (k[e] != 0) {
        ++nz;
        const uint32_t z = ((uint32_t)k[e] << 1) ^ (uint32_t)(k[e] >> 31);
        if (z > kmx) kmx = z;
      }
    if (nz != ncorr || nbits(kmx) != wk) return OR_ERR_CORRUPT;
  } else if (wk > 0 && dense) {
    for (int64_t e = 0; e < N; ++e) {
      const uint32_t z = get_bits(cw, (uint64_t)e * wk, wk);
      k[e] = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
    }
  } else if (wk > 0) {
    int64_t prev = -1;
    for (int64_t ci = 0; ci < ncorr; ++ci) {
      const uint64_t pos = (uint64_t)ci * (ib + wk);
      const int64_t e = get_bits(cw, pos, ib);
      const uint32_t z = get_bits(cw, pos + ib, wk);
      if (e >= N || e <= prev) return OR_ERR_CORRUPT;     /* increasing element order */
      k[e] = (int32_t)((z >> 1) ^ (0u - (z & 1u)));
      prev = e;
    }
  }
  int64_t prev = -1;
  for (int64_t i = 0; i < nesc; ++i) {
    const int64_t e = rd32(rec + off_ei + 4 * i);
    if (e >= N || e <= prev) return OR_ERR_CORRUPT;
    esc[e] = 1;
    escval[e] = get_val(rec + off_ev + i * es, dtype);
    prev = e;
  }
  *r_out = r;
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Coefficients as the FP32 (mixed-precision) form defines them, so     */
/* that its quantized codes can be compared code for code: the          */
/* projection of Sec. 2.5 Eq. 5 evaluated in binary32 on a shifted row, */
/*   d_j = fl(x_j - x_0),  s_m = fma chain over j = m, m+4, ... (m < 4), */
/*   c = fma(x_0, vsum_k, fl(fl(s_0 + s_1) + fl(s_2 + s_3))),           */
/* with vsum_k = fl32(sum_j Vst[j][k]) summed in double, j ascending.   */
/* The FP64-semantics quantizer (or_quantize on these values) then      */
/* takes the same decision as the kernel.  C is L x r (leading r).      */
/* ------------------------------------------------------------------ */
void or_project_f32(const double* A, int64_t L, int n, const double* Vst, int r, double* C) {
  for (int k = 0; k < r; ++k) {
    double cs = 0.0;
    for (int j = 0; j < n; ++j) cs += (double)(float)Vst[j * r + k];
    const float vsum = (float)cs;
    for (int64_t l = 0; l < L; ++l) {
      const float a0 = (float)A[l * n];
      float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int j = 0; j < n; ++j) {
        const float d = (float)A[l * n + j] - a0;
        s[j & 3] = fmaf(d, (float)Vst[j * r + k], s[j & 3]);
      }
      const float sum = (s[0] + s[1]) + (s[2] + s[3]);
      C[l * r + k] = (double)fmaf(a0, vsum, sum);
    }
  }
}
