// Plain FP64 compression path: one CTA per block.
//
// Per block (Algorithm 1 step 3 of arXiv 2601.20113, with the readings of the
// pointwise-bound form):
//   Gram G = A^T A (cross-product SVD, Sec. 2.7.1)      FP64, sequential fma per entry
//   Jacobi eigensolve, round-robin ordering (Sec. 2.3)   FP64, one warp, lane = row
//   projection C = A Vst (Sec. 2.5, Eq. 5)               FP64 fma chain per coefficient
//   quantization q = rint(C / delta)
//   bisection for the smallest rank with E(r) <= eps_l^2 (Sec. 2.4 Eq. 4, Eq. 6)
//   pointwise correction k = rint((x - xhat) / 2eb), escapes
//   per-block record size (raw if not smaller)
// Every floating-point operation that decides a stored value is written with
// an explicit rounding intrinsic, in the same order as the definitions, so the
// result is bit-identical to any IEEE implementation of those definitions.
#include "dls_internal.cuh"

namespace dls {
namespace {

constexpr int kThreads = 256;
constexpr int kRC = 256;  // rows per staged chunk of the Gram pass

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T> __device__ __forceinline__ double to_dt(double x);
template <> __device__ __forceinline__ double to_dt<float>(double x) { return (double)__double2float_rn(x); }
template <> __device__ __forceinline__ double to_dt<double>(double x) { return x; }

// Dequantized coefficient in the field dtype: dtype(q) * dtype(delta).
template <typename T> __device__ __forceinline__ T dequant(int32_t q, T delta_t);
template <> __device__ __forceinline__ float dequant<float>(int32_t q, float d) { return __fmul_rn(__int2float_rn(q), d); }
template <> __device__ __forceinline__ double dequant<double>(int32_t q, double d) { return __dmul_rn((double)q, d); }
template <typename T> __device__ __forceinline__ T tfma(T a, T b, T c);
template <> __device__ __forceinline__ float tfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double tfma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int NM>
struct Smem {
  double G[NM * NM], H[NM * NM], G2[NM * NM], V[NM * NM];
  double Vst[NM * NM];      // n x rcap, leading dimension rcap, dtype-rounded values
  double buf[kThreads * NM];// Gram chunk (kRC x n) or E chunk partials (kThreads x n)
  double colsum[NM];
  double cc[NM / 2], ss[NM / 2], tt[NM / 2];
  int pp[NM / 2], qq[NM / 2], act[NM / 2];
  int rowpair[NM];
  double Ecur;
  int ovf, nonfinite;
  int wq[NM];
  int ncorr, nesc, kmax;
};

// Round-robin pairing (circle method) of m indices, round `round`, pair i.
__device__ __forceinline__ void rr_pair(int round, int i, int m, int& p, int& q) {
  int a, b;
  if (i == 0) { a = m - 1; b = round; }
  else { a = (round + i) % (m - 1); b = (round - i + (m - 1)) % (m - 1); }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Jacobi eigensolve of S.G (n x n) by warp 0; eigenvectors in S.V (unsorted),
// eigenvalues on the diagonal of S.G.  Mirrors the definition step by step:
// rotations of a round are computed from the matrix at the start of the round,
// rows are rotated, then columns, the upper triangle is mirrored, and the
// rotated pairs get their closed-form diagonal and a zero off-diagonal.
template <int NM>
__device__ void jacobi_warp(Smem<NM>& S, int n, int lane) {
  double* G = S.G;
  double* H = S.H;
  double* G2 = S.G2;
  double* V = S.V;
  if (lane < n)
    for (int b = 0; b < n; ++b) V[lane * n + b] = (lane == b) ? 1.0 : 0.0;
  double tr = 0.0;
  if (lane == 0)
    for (int i = 0; i < n; ++i) tr = dadd(tr, G[i * n + i]);
  tr = __shfl_sync(0xffffffffu, tr, 0);
  const double tol = dmul(1e-15, tr);
  const int m = n + (n & 1);
  __syncwarp();
  for (int sweep = 0; sweep < 30 && n > 1; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < m - 1; ++round) {
      if (lane < n) S.rowpair[lane] = -1;
      __syncwarp();
      int act = 0;
      if (lane < m / 2) {
        int p, q;
        rr_pair(round, lane, m, p, q);
        S.pp[lane] = p;
        S.qq[lane] = q;
        if (q < n) {
          double apq = G[p * n + q];
          if (fabs(apq) > tol) {
            double theta = ddiv(dsub(G[q * n + q], G[p * n + p]), dmul(2.0, apq));
            double t;
            if (fabs(theta) > 1e150) t = ddiv(0.5, theta);
            else t = ddiv(theta >= 0.0 ? 1.0 : -1.0, dadd(fabs(theta), __dsqrt_rn(dadd(1.0, dmul(theta, theta)))));
            double c = ddiv(1.0, __dsqrt_rn(dadd(1.0, dmul(t, t))));
            S.cc[lane] = c;
            S.ss[lane] = dmul(t, c);
            S.tt[lane] = t;
            act = 1;
            S.rowpair[p] = lane;
            S.rowpair[q] = lane;
          }
        }
        S.act[lane] = act;
      }
      rotated += __popc(__ballot_sync(0xffffffffu, act));
      __syncwarp();
      // rows: H = J^T G
      if (lane < n) {
        const int a = lane;
        const int i = S.rowpair[a];
        if (i >= 0) {
          const int p = S.pp[i], q = S.qq[i];
          const double c = S.cc[i], s = S.ss[i];
          if (a == p)
            for (int b = 0; b < n; ++b) H[a * n + b] = dsub(dmul(c, G[p * n + b]), dmul(s, G[q * n + b]));
          else
            for (int b = 0; b < n; ++b) H[a * n + b] = dadd(dmul(s, G[p * n + b]), dmul(c, G[q * n + b]));
        } else {
          for (int b = 0; b < n; ++b) H[a * n + b] = G[a * n + b];
        }
      }
      __syncwarp();
      // columns: G2 = H J, upper triangle, mirrored
      if (lane < n) {
        const int a = lane;
        for (int b = a; b < n; ++b) {
          const int i = S.rowpair[b];
          double v;
          if (i >= 0) {
            const int p = S.pp[i], q = S.qq[i];
            const double c = S.cc[i], s = S.ss[i];
            if (b == p) v = dsub(dmul(c, H[a * n + p]), dmul(s, H[a * n + q]));
            else v = dadd(dmul(s, H[a * n + p]), dmul(c, H[a * n + q]));
          } else {
            v = H[a * n + b];
          }
          G2[a * n + b] = v;
          G2[b * n + a] = v;
        }
      }
      __syncwarp();
      if (lane < m / 2 && S.act[lane]) {
        const int p = S.pp[lane], q = S.qq[lane];
        const double t = S.tt[lane], gpq = G[p * n + q];
        G2[p * n + p] = dsub(G[p * n + p], dmul(t, gpq));
        G2[q * n + q] = dadd(G[q * n + q], dmul(t, gpq));
        G2[p * n + q] = 0.0;
        G2[q * n + p] = 0.0;
      }
      if (lane < n) {
        const int a = lane;
        for (int i = 0; i < m / 2; ++i) {
          if (!S.act[i]) continue;
          const int p = S.pp[i], q = S.qq[i];
          const double c = S.cc[i], s = S.ss[i];
          const double vp = V[a * n + p], vq = V[a * n + q];
          V[a * n + p] = dsub(dmul(c, vp), dmul(s, vq));
          V[a * n + q] = dadd(dmul(s, vp), dmul(c, vq));
        }
      }
      __syncwarp();
      if (lane < n)
        for (int b = 0; b < n; ++b) G[lane * n + b] = G2[lane * n + b];
      __syncwarp();
    }
    if (rotated == 0) break;
  }
}

// Stable descending order of the clamped eigenvalues, sign-normalised
// columns, first rcap columns rounded to the dtype into S.Vst.
template <typename T, int NM>
__device__ void sort_and_store(Smem<NM>& S, int n, int rcap, int lane, double* vst_out) {
  if (lane < n) {
    const int k = lane;
    double dk = S.G[k * n + k];
    dk = dk < 0.0 ? 0.0 : dk;
    int pos = 0;
    for (int j = 0; j < n; ++j) {
      double dj = S.G[j * n + j];
      dj = dj < 0.0 ? 0.0 : dj;
      if (dj > dk || (dj == dk && j < k)) ++pos;
    }
    int imax = 0;
    double amax = -1.0;
    for (int a = 0; a < n; ++a) {
      double av = fabs(S.V[a * n + k]);
      if (av > amax) { amax = av; imax = a; }
    }
    const bool neg = S.V[imax * n + k] < 0.0;
    if (pos < rcap) {
      for (int a = 0; a < n; ++a) {
        double v = S.V[a * n + k];
        v = neg ? -v : v;
        const double vs = to_dt<T>(v);
        S.Vst[a * rcap + pos] = vs;
        vst_out[a * rcap + pos] = vs;
      }
    }
  }
}

// E(r) = sum (A - D_r)^2 in the fixed order: per column, rows in chunks of 32
// (sequential fma), chunk sums in order, then column sums in order.
// D_r is the decode contract: fma chain over k < r in the field dtype.
template <typename T, int NM>
__device__ double block_err(Smem<NM>& S, const Plan& P, const Geom& g, const T* __restrict__ in,
                            const int32_t* __restrict__ q, int n, int64_t L, int r, int ld, T delta_t) {
  const int tid = threadIdx.x;
  const int64_t nch = cdiv(L, 32);
  if (tid < n) S.colsum[tid] = 0.0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nch; c0 += kThreads) {
    const int64_t c = c0 + tid;
    if (c < nch) {
      double pc[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) pc[j] = 0.0;
      const int64_t l1 = (c + 1) * 32 < L ? (c + 1) * 32 : L;
      for (int64_t l = c * 32; l < l1; ++l) {
        T ch[NM];
#pragma unroll
        for (int k = 0; k < NM; ++k) ch[k] = (k < r) ? dequant<T>(q[(int64_t)k * L + l], delta_t) : T(0);
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < NM; ++k)
              if (k < r) acc = tfma<T>(ch[k], (T)S.Vst[j * ld + k], acc);
            const double d = dsub((double)in[a_index(P, g, l, j)], (double)acc);
            pc[j] = dfma(d, d, pc[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NM; ++j)
        if (j < n) S.buf[(c - c0) * n + j] = pc[j];
    }
    __syncthreads();
    if (tid < n) {
      const int64_t cend = (nch - c0) < kThreads ? (nch - c0) : kThreads;
      double s = S.colsum[tid];
      for (int64_t cc = 0; cc < cend; ++cc) s = dadd(s, S.buf[cc * n + tid]);
      S.colsum[tid] = s;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double E = 0.0;
    for (int j = 0; j < n; ++j) E = dadd(E, S.colsum[j]);
    S.Ecur = E;
  }
  __syncthreads();
  return S.Ecur;
}

template <typename T, int NM>
__global__ void __launch_bounds__(kThreads) k_plain(Plan P, const T* __restrict__ in, Work W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<NM>& S = *reinterpret_cast<Smem<NM>*>(smem_raw);
  const int64_t bi = blockIdx.x;
  const Geom g = block_geom(P, P.b0 + bi);
  const VarInfo vi = W.vars[g.v];
  const int n = g.n;
  const int64_t L = g.L, N = g.N;
  const int rcap = P.rank_cap < n ? P.rank_cap : n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T delta_t = (T)to_dt<T>(vi.delta);

  if (tid == 0) { S.ovf = 0; S.nonfinite = 0; S.ncorr = 0; S.nesc = 0; S.kmax = 0; }
  if (tid < NM) S.wq[tid] = 0;

  // ---- 1. Gram: G[i][j] = sum_l A[l][i] A[l][j], sequential fma over l
  const int npairs = n * (n + 1) / 2;
  constexpr int kPairsPerThread = (NM * (NM + 1) / 2 + kThreads - 1) / kThreads;
  double acc[kPairsPerThread];
  int pi[kPairsPerThread], pj[kPairsPerThread];
#pragma unroll
  for (int s = 0; s < kPairsPerThread; ++s) {
    acc[s] = 0.0;
    int idx = tid + s * kThreads;
    pi[s] = -1; pj[s] = -1;
    if (idx < npairs) {
      int i = 0;
      while (idx >= n - i) { idx -= n - i; ++i; }
      pi[s] = i; pj[s] = i + idx;
    }
  }
  int nonfinite = 0;
  for (int64_t l0 = 0; l0 < L; l0 += kRC) {
    const int rows = (int)((L - l0) < kRC ? (L - l0) : kRC);
    for (int e = tid; e < rows * n; e += kThreads) {
      const int j = e / rows, lr = e - j * rows;
      const double x = (double)in[a_index(P, g, l0 + lr, j)];
      if (!isfinite(x)) nonfinite = 1;
      S.buf[lr * n + j] = x;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kPairsPerThread; ++s) {
      if (pi[s] >= 0) {
        const int i = pi[s], j = pj[s];
        double a = acc[s];
        for (int lr = 0; lr < rows; ++lr) a = dfma(S.buf[lr * n + i], S.buf[lr * n + j], a);
        acc[s] = a;
      }
    }
    __syncthreads();
  }
  if (nonfinite) S.nonfinite = 1;
#pragma unroll
  for (int s = 0; s < kPairsPerThread; ++s)
    if (pi[s] >= 0) { S.G[pi[s] * n + pj[s]] = acc[s]; S.G[pj[s] * n + pi[s]] = acc[s]; }
  __syncthreads();
  if (S.nonfinite) {
    if (tid == 0) atomicOr(&W.status->nonfinite, 1u);
    return;
  }

  // ---- 2. eigensolve (warp 0) and stored basis; with a fixed basis of this
  // Gram order (Sec. 4), its first rcap modes in the given order instead
  double* vst_out = W.vst + bi * (int64_t)P.nmax * P.nmax;
  if (W.basis && n == P.basis_n) {
    for (int e = tid; e < n * rcap; e += kThreads) {
      const int a = e / rcap, k = e - a * rcap;
      const double vs = to_dt<T>(W.basis[a * n + k]);
      S.Vst[a * rcap + k] = vs;
      vst_out[a * rcap + k] = vs;
    }
  } else if (warp == 0) {
    jacobi_warp<NM>(S, n, lane);
    __syncwarp();
    sort_and_store<T, NM>(S, n, rcap, lane, vst_out);
  }
  __syncthreads();

  // ---- 3. projection and quantization: q[k][l] = rint((sum_j A[l][j] Vst[j][k]) / delta)
  int32_t* qb = W.q + (g.pt_off - P.pt_base);
  const double qlim = (sizeof(T) == 4) ? kQmaxF32 : kQmaxF64;
  int ovf = 0;
  for (int64_t l = tid; l < L; l += kThreads) {
    double a[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) a[j] = (j < n) ? (double)in[a_index(P, g, l, j)] : 0.0;
    for (int k = 0; k < rcap; ++k) {
      double c = 0.0;
#pragma unroll
      for (int j = 0; j < NM; ++j)
        if (j < n) c = dfma(a[j], S.Vst[j * rcap + k], c);
      const double y = ddiv(c, vi.delta);
      int32_t qv = 0;
      if (!(fabs(y) < qlim)) ovf = 1;
      else qv = (int32_t)rint(y);
      qb[(int64_t)k * L + l] = qv;
    }
  }
  if (ovf) S.ovf = 1;
  __syncthreads();
  const bool overflow = S.ovf != 0;

  // ---- 4. rank: bisection on pass(r) <=> E(r) <= eps_l^2
  const double el2 = (P.eb_type == DLS_EB_NRMSE)
                         ? dmul(dmul(vi.eb, vi.eb), ddiv((double)N, P.kbound))
                         : dmul(dmul(vi.eb, vi.eb), (double)N);
  int r = 0, nprobes = 0;
  bool raw = overflow;
  if (!raw) {
    int lo = 0, hi = rcap;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const double E = block_err<T, NM>(S, P, g, in, qb, n, L, mid, rcap, delta_t);
      ++nprobes;
      if (E <= el2) hi = mid; else lo = mid + 1;
    }
    r = lo;
    if (P.eb_type == DLS_EB_NRMSE) {
      const double E = block_err<T, NM>(S, P, g, in, qb, n, L, r, rcap, delta_t);
      if (!(E <= el2)) raw = true;
    }
  }

  // ---- 5. pointwise correction at r, and per-block widths
  int32_t* kb = W.kc + (g.pt_off - P.pt_base);
  if (!raw && P.eb_type != DLS_EB_NRMSE) {
    const double eb = vi.eb, step = vi.step;
    const T step_t = (T)to_dt<T>(step);
    int nc = 0, ne = 0;
    uint32_t kmx = 0;
    uint32_t qmx[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) qmx[k] = 0;
    for (int64_t l = tid; l < L; l += kThreads) {
      T ch[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        int32_t qv = (k < r) ? qb[(int64_t)k * L + l] : 0;
        if (k < r) { uint32_t z = zigzag(qv); qmx[k] = z > qmx[k] ? z : qmx[k]; }
        ch[k] = (k < r) ? dequant<T>(qv, delta_t) : T(0);
      }
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        if (j < n) {
          T xh = T(0);
#pragma unroll
          for (int k = 0; k < NM; ++k)
            if (k < r) xh = tfma<T>(ch[k], (T)S.Vst[j * rcap + k], xh);
          const double x = (double)in[a_index(P, g, l, j)];
          const double R = dsub(x, (double)xh);
          const double y = ddiv(R, step);
          const double kk = rint(y);
          int32_t kv = 0;
          bool esc = false;
          double xt;
          if (kk == 0.0) {
            xt = (double)xh;
          } else if (fabs(kk) > kKmax) {
            esc = true;
            xt = 0.0;
          } else {
            xt = (double)tfma<T>((T)kk, step_t, xh);
          }
          if (!esc && fabs(dsub(x, xt)) > eb) esc = true;
          if (esc) { kv = kEscape; ++ne; }
          else if (kk != 0.0) {
            kv = (int32_t)kk;
            ++nc;
            uint32_t z = zigzag(kv);
            kmx = z > kmx ? z : kmx;
          }
          kb[a_elem(g, l, j)] = kv;
        }
      }
    }
    // block reductions
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nc += __shfl_xor_sync(0xffffffffu, nc, o);
      ne += __shfl_xor_sync(0xffffffffu, ne, o);
      kmx = max(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      uint32_t v = qmx[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
      qmx[k] = v;
    }
    if (lane == 0) {
      atomicAdd(&S.ncorr, nc);
      atomicAdd(&S.nesc, ne);
      atomicMax(&S.kmax, (int)kmx);
#pragma unroll
      for (int k = 0; k < NM; ++k) if (k < r) atomicMax(&S.wq[k], bit_width(qmx[k]));
    }
  } else if (!raw) {
    // NRMSE mode: no corrections, widths only
    uint32_t qmx[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) qmx[k] = 0;
    for (int64_t l = tid; l < L; l += kThreads) {
#pragma unroll
      for (int k = 0; k < NM; ++k)
        if (k < r) { uint32_t z = zigzag(qb[(int64_t)k * L + l]); qmx[k] = z > qmx[k] ? z : qmx[k]; }
    }
    for (int64_t e = tid; e < N; e += kThreads) kb[e] = 0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      uint32_t v = qmx[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0 && k < r) atomicMax(&S.wq[k], bit_width(v));
    }
  }
  __syncthreads();

  // ---- 6. record size (raw when the encoded record is not smaller)
  if (tid == 0) {
    BlockMeta m;
    const int es = (int)sizeof(T);
    const int64_t rawsz = raw_record_bytes(N, es);
    m.rcap = rcap;
    m.nprobes = nprobes;
    m.r = 0; m.wk = 0; m.ib = 0; m.ncorr = 0; m.nesc = 0;
    m.flags = g.side ? (int)kFlagSpatial : 0;
    for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
    if (!raw) {
      for (int k = 0; k < r; ++k) m.wq[k] = (uint8_t)S.wq[k];
      const int wk = bit_width((uint32_t)S.kmax);
      const int ib = bit_width((uint32_t)(N - 1));
      const RecLayout lay = rec_layout(r, n, L, N, es, m.wq, wk, ib, S.ncorr, S.nesc);
      if (lay.size >= rawsz) {
        raw = true;
      } else {
        m.r = r; m.wk = wk; m.ib = ib; m.ncorr = S.ncorr; m.nesc = S.nesc;
        m.flags |= lay.dense ? (int)kFlagDense : 0;
        m.nbytes = lay.size;
      }
    }
    if (raw) {
      m.r = 0; m.wk = 0; m.ib = 0; m.ncorr = 0; m.nesc = 0;
      for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
      m.flags = (int)kFlagRaw | (g.side ? (int)kFlagSpatial : 0);
      m.nbytes = rawsz;
    }
    W.meta[bi] = m;
  }
}

template <typename T, int NM>
int launch_t(const Plan& p, const void* d_in, const Work& w, cudaStream_t s) {
  const size_t smem = sizeof(Smem<NM>);
  cudaError_t e = cudaFuncSetAttribute(k_plain<T, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return DLS_ERR_CUDA;
  if (p.nb == 0) return DLS_OK;
  k_plain<T, NM><<<(unsigned)p.nb, kThreads, smem, s>>>(p, (const T*)d_in, w);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

}  // namespace

int launch_plain_compress(const Plan& p, const void* d_in, const Work& w, cudaStream_t s) {
  if (p.dtype == DLS_F32) {
    if (p.nmax <= 16) return launch_t<float, 16>(p, d_in, w, s);
    return launch_t<float, 32>(p, d_in, w, s);
  }
  if (p.nmax <= 16) return launch_t<double, 16>(p, d_in, w, s);
  return launch_t<double, 32>(p, d_in, w, s);
}

}  // namespace dls
