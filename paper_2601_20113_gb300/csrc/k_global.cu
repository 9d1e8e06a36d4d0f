// Global-basis mode (Algorithm 1 of arXiv 2601.20113 as stated: one basis per
// variable, learned from random patches of the first snapshot, Sec. 2.3
// Eq. 2-3; per patch of every snapshot the coefficients on it, Sec. 2.5
// Eq. 5, the largest-magnitude prefix meeting the local tolerance of Sec. 2.4
// Eq. 4 found by bisection, Eq. 6; reconstruction, Sec. 2.6).  FP64
// throughout, so that every stored decision is the definition's; the device
// steps are
//   k_gb_sample   the sample matrix Q (S x M) from the first snapshot,
//   k_gb_gram     G = Q^T Q, each entry a sequential sum over the samples,
//   k_gb_jacobi   the eigenvectors of G by cyclic Jacobi in one CTA (G and,
//                 when they fit, V in shared memory), sorted by decreasing
//                 eigenvalue and signed (largest component positive),
//   k_gb_norm     ||u||^2 of the variable, then eps_l^2 and delta,
//   k_gb_patch    a warp per patch: alpha = Phi^T u, q = rint(alpha / delta),
//                 the magnitude order, the bisection on the kept count, the
//                 record into the patch's slot,
//   scan + copy   the record offsets and the stream.
// The decoder rebuilds each patch from its kept modes in kept order.
#include "dls_device.cuh"

namespace dls {
namespace {

constexpr int kGbMaxM = 128;
constexpr int kGbHdr = 80;
constexpr uint32_t kGbMagic = 0x47534C44u;   // "DLSG"
constexpr int kGbWarps = 8;                  // patches in flight per CTA
constexpr int kGbStatCtas = 512;

struct GbPlan {
  int64_t dims[4];
  int px, py, pz, M, ib;
  int64_t S, K, nrec, npx, npy, npz;
  double eps_t;
  int64_t slot_bytes;          // a patch's record slot (largest record, 16-aligned)
  int64_t offsets_pos, payload_pos;
};

struct GbStatus {
  unsigned int bad_origin, overflow, corrupt, nonfinite;
  double eps_l2, delta;
  unsigned long long total;
};

__host__ __device__ inline int gb_width(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Largest record of a patch: n = M entries of ib + 63 bits.
__host__ __device__ inline int64_t gb_record_max(int M, int ib) {
  const int64_t words = ((int64_t)M * (ib + 63) + 31) / 32;
  return align_up(8 + 4 * words, 8);
}

int gb_make_plan(const dls_gb_params* p, GbPlan* g) {
  if (!p) return DLS_ERR_INVALID_ARG;
  memset(g, 0, sizeof(*g));
  for (int a = 0; a < 4; ++a) {
    if (p->dims[a] < 1) return DLS_ERR_INVALID_ARG;
    g->dims[a] = p->dims[a];
  }
  if (p->m < 1 || !(p->eps_t > 0.0) || !isfinite(p->eps_t) || p->nsample < 1) return DLS_ERR_INVALID_ARG;
  g->px = g->py = p->m;
  g->pz = p->dims[2] > 1 ? p->m : 1;
  const int64_t M = (int64_t)g->px * g->py * g->pz;
  if (M > kGbMaxM) return DLS_ERR_INVALID_ARG;
  g->M = (int)M;
  if (p->dims[0] % g->px || p->dims[1] % g->py || p->dims[2] % g->pz) return DLS_ERR_INVALID_ARG;
  g->ib = gb_width((uint64_t)(M - 1));
  g->S = p->nsample;
  g->K = p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  g->npx = p->dims[0] / g->px;
  g->npy = p->dims[1] / g->py;
  g->npz = p->dims[2] / g->pz;
  g->nrec = g->npx * g->npy * g->npz * p->dims[3];
  g->eps_t = p->eps_t;
  g->slot_bytes = align_up(gb_record_max(g->M, g->ib), 16);
  g->offsets_pos = kGbHdr + 8 * M * M;
  g->payload_pos = g->offsets_pos + 8 * (g->nrec + 1);
  return DLS_OK;
}

struct GbLayout {
  size_t Q, G, V, phi, lam, partial, status, sizes, offsets, slots, total;
};

GbLayout gb_layout(const GbPlan& g) {
  GbLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (size_t)align_up((int64_t)(off + bytes), 256);
    return o;
  };
  const size_t MM = (size_t)g.M * g.M;
  const size_t me = (size_t)(g.M + (g.M & 1));   // the Jacobi's even order
  L.Q = take(sizeof(double) * (size_t)g.S * g.M);
  L.G = take(sizeof(double) * MM);
  L.V = take(sizeof(double) * me * me);
  L.phi = take(sizeof(double) * MM);
  L.lam = take(sizeof(double) * (size_t)g.M);
  L.partial = take(sizeof(double) * kGbStatCtas);
  L.status = take(sizeof(GbStatus));
  L.sizes = take(sizeof(unsigned long long) * (size_t)(g.nrec + 1));
  L.offsets = take(sizeof(unsigned long long) * (size_t)(g.nrec + 1));
  L.slots = take((size_t)g.slot_bytes * (size_t)g.nrec);
  L.total = off;
  return L;
}

// ---------------------------------------------------------------- step 1: the basis
// Row s of Q: the patch of the first snapshot at origins[s] (x fastest).
__global__ void k_gb_sample(GbPlan g, const float* __restrict__ in, const int64_t* __restrict__ origins, double* Q,
                            GbStatus* st) {
  const int64_t s = blockIdx.x;
  const int64_t x0 = origins[3 * s], y0 = origins[3 * s + 1], z0 = origins[3 * s + 2];
  if (x0 < 0 || y0 < 0 || z0 < 0 || x0 + g.px > g.dims[0] || y0 + g.py > g.dims[1] || z0 + g.pz > g.dims[2]) {
    if (threadIdx.x == 0) atomicOr(&st->bad_origin, 1u);
    return;
  }
  for (int i = threadIdx.x; i < g.M; i += blockDim.x) {
    const int ix = i % g.px, iy = (i / g.px) % g.py, iz = i / (g.px * g.py);
    Q[s * g.M + i] = (double)in[((z0 + iz) * g.dims[1] + (y0 + iy)) * g.dims[0] + (x0 + ix)];
  }
}

// G[i][j] = sum_s Q[s][i] Q[s][j], one entry a thread, samples in order (fma).
__global__ void k_gb_gram(GbPlan g, const double* __restrict__ Q, double* G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.M * g.M) return;
  const int i = e / g.M, j = e - i * g.M;
  double acc = 0.0;
  for (int64_t s = 0; s < g.S; ++s) acc = __fma_rn(Q[s * g.M + i], Q[s * g.M + j], acc);
  G[e] = acc;
}

__device__ __forceinline__ void gb_pair(int round, int i, int m, int& p, int& q) {
  int a, b;
  if (i == 0) { a = m - 1; b = round; }
  else { a = (round + i) % (m - 1); b = (round - i + (m - 1)) % (m - 1); }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Cyclic Jacobi of G (order M, padded with a zero row and column to even m),
// one CTA: every round rotates the m/2 disjoint pairs of the round-robin
// circle whose off-diagonal entry exceeds 2^-53 sqrt(|a_pp a_qq|); each 2 x 2
// block of A (pair k's rows, pair l's columns) becomes J_k^T A_kl J_l, with
// the exact 2 x 2 result on the diagonal blocks, and V's column pairs rotate.
// Stops after a sweep without rotation (50 sweeps at most).  Then the modes:
// columns of V by decreasing eigenvalue (index order on ties), each signed so
// that its largest-magnitude component (the first on ties) is positive.
constexpr int kJacThreads = 1024;
__global__ void __launch_bounds__(kJacThreads, 1) k_gb_jacobi(GbPlan g, const double* __restrict__ G, double* Vg,
                                                               double* phi, double* lam_out, int v_shared) {
  extern __shared__ double A[];               // m x m, then V (m x m) when v_shared
  __shared__ int pq[kGbMaxM / 2];
  __shared__ double jc[kGbMaxM / 2], js[kGbMaxM / 2], jt[kGbMaxM / 2];
  __shared__ double lam[kGbMaxM];
  __shared__ int order[kGbMaxM];
  const int tid = threadIdx.x;
  const int M = g.M, m = M + (M & 1), h = m / 2;
  double* V = v_shared ? A + m * m : Vg;
  for (int e = tid; e < m * m; e += kJacThreads) {
    const int i = e / m, j = e - i * m;
    A[e] = (i < M && j < M) ? G[i * M + j] : 0.0;
    V[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 50 && M > 1; ++sweep) {
    int any = 0;
    for (int round = 0; round < m - 1; ++round) {
      int act = 0;
      if (tid < h) {
        int p, q;
        gb_pair(round, tid, m, p, q);
        const double app = A[p * m + p], aqq = A[q * m + q], apq = A[p * m + q];
        double c = 1.0, s = 0.0, t = 0.0;
        if (apq != 0.0 && fabs(apq) > 0x1p-53 * sqrt(fabs(app) * fabs(aqq))) {
          const double theta = (aqq - app) / (2.0 * apq);
          if (fabs(theta) > 1e150) t = 0.5 / theta;
          else t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
          act = 1;
        }
        pq[tid] = p | q << 8 | act << 16;
        jc[tid] = c;
        js[tid] = s;
        jt[tid] = t;
      }
      if (!__syncthreads_or(act)) continue;
      any = 1;
      for (int it = tid; it < h * h + m * h; it += kJacThreads) {
        if (it < h * h) {
          const int k = it / h, l = it - k * h;
          const int a = pq[k], b = pq[l];
          if (!((a | b) >> 16)) continue;
          const int p = a & 255, q = (a >> 8) & 255, pp = b & 255, qq = (b >> 8) & 255;
          const double ck = jc[k], sk = js[k], cl = jc[l], sl = js[l];
          if (k == l) {
            const double t = jt[k], apq = A[p * m + q];
            const double np = A[p * m + p] - t * apq, nq = A[q * m + q] + t * apq;
            A[p * m + p] = np;
            A[q * m + q] = nq;
            A[p * m + q] = 0.0;
            A[q * m + p] = 0.0;
            continue;
          }
          const double x = A[p * m + pp], y = A[p * m + qq], z = A[q * m + pp], w = A[q * m + qq];
          const double r1 = ck * x - sk * z, r2 = ck * y - sk * w, r3 = sk * x + ck * z, r4 = sk * y + ck * w;
          A[p * m + pp] = cl * r1 - sl * r2;
          A[p * m + qq] = sl * r1 + cl * r2;
          A[q * m + pp] = cl * r3 - sl * r4;
          A[q * m + qq] = sl * r3 + cl * r4;
        } else {
          const int it2 = it - h * h;
          const int i = it2 / h, l = it2 - i * h;
          const int b = pq[l];
          if (!(b >> 16)) continue;
          const int p = b & 255, q = (b >> 8) & 255;
          const double c = jc[l], s = js[l];
          const double x = V[i * m + p], y = V[i * m + q];
          V[i * m + p] = c * x - s * y;
          V[i * m + q] = s * x + c * y;
        }
      }
      __syncthreads();
    }
    if (!any) break;
  }
  for (int k = tid; k < M; k += kJacThreads) lam[k] = A[k * m + k];
  __syncthreads();
  for (int k = tid; k < M; k += kJacThreads) {
    int rank = 0;
    for (int j = 0; j < M; ++j) rank += (lam[j] > lam[k] || (lam[j] == lam[k] && j < k)) ? 1 : 0;
    order[rank] = k;
  }
  __syncthreads();
  for (int r = tid; r < M; r += kJacThreads) {
    const int k = order[r];
    int imax = 0;
    double vmax = -1.0;
    for (int i = 0; i < M; ++i) {
      const double a = fabs(V[i * m + k]);
      if (a > vmax) { vmax = a; imax = i; }
    }
    const double sg = V[imax * m + k] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < M; ++i) phi[i * M + r] = sg * V[i * m + k];
    lam_out[r] = lam[k];
  }
}

// ---------------------------------------------------------------- step 2: the tolerance
// CTA c sums u^2 over a fixed contiguous range in a fixed order.
__global__ void __launch_bounds__(256) k_gb_norm(GbPlan g, const float* __restrict__ in, double* partial,
                                                 GbStatus* st) {
  const int64_t per = cdiv(g.K, kGbStatCtas);
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = (i0 + per) < g.K ? i0 + per : g.K;
  double s = 0.0;
  int bad = 0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
    const double x = (double)in[i];
    if (!isfinite(x)) bad = 1;
    s = __fma_rn(x, x, s);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
  if (bad) atomicOr(&st->nonfinite, 1u);
}

// eps = eps_t ||u|| / 100, eps_l^2 = eps^2 M / K, delta = eps / sqrt(K).
__global__ void k_gb_resolve(GbPlan g, const double* partial, GbStatus* st) {
  double s2 = 0.0;
  for (int c = 0; c < kGbStatCtas; ++c) s2 = __dadd_rn(s2, partial[c]);
  const double eps = __ddiv_rn(__dmul_rn(g.eps_t, __dsqrt_rn(s2)), 100.0);
  st->eps_l2 = __ddiv_rn(__dmul_rn(__dmul_rn(eps, eps), (double)g.M), (double)g.K);
  st->delta = __ddiv_rn(eps, __dsqrt_rn((double)g.K));
}

// ---------------------------------------------------------------- step 3: the patches
// Per warp in shared memory (after the basis, M x M doubles, [component][mode]).
struct GbWarp {
  double u[kGbMaxM];
  double al[kGbMaxM];
  double qd[kGbMaxM];          // q_k delta, by mode
  long long q[kGbMaxM];
  int ord[kGbMaxM];            // modes by decreasing |alpha| (index order on ties)
  uint32_t words[((kGbMaxM * 70 + 31) / 32) + 4];
};

__host__ __device__ inline size_t gb_patch_smem(int M) {
  return sizeof(double) * (size_t)M * M + sizeof(GbWarp) * kGbWarps;
}

__device__ __forceinline__ uint64_t gb_zz(long long q) { return ((uint64_t)q << 1) ^ (uint64_t)(q >> 63); }

// OR `width` (<= 64) bits of v into the words from bit pos (shared memory).
__device__ __forceinline__ void gb_put(uint32_t* w, uint64_t pos, uint64_t v, int width) {
  for (int done = 0; done < width;) {
    const int sh = (int)(pos & 31);
    const int take = (32 - sh) < (width - done) ? (32 - sh) : (width - done);
    const uint32_t part = (uint32_t)((v >> done) & ((take == 32) ? 0xFFFFFFFFull : ((1ull << take) - 1ull)));
    atomicOr(&w[pos >> 5], part << sh);
    pos += (uint64_t)take;
    done += take;
  }
}

__device__ __forceinline__ double gb_warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// A warp per patch, patches in (t, z, y, x) order over the grid's warps.
__global__ void __launch_bounds__(kGbWarps * 32) k_gb_patch(GbPlan g, const float* __restrict__ in,
                                                            const double* __restrict__ phi_g, const GbStatus* stc,
                                                            GbStatus* st, unsigned long long* sizes, uint8_t* slots) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int M = g.M;
  double* phi = reinterpret_cast<double*>(gsm);
  GbWarp& W = reinterpret_cast<GbWarp*>(gsm + sizeof(double) * (size_t)M * M)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) phi[e] = phi_g[e];
  __syncthreads();
  const double eps_l2 = stc->eps_l2, delta = stc->delta;
  const int ib = g.ib;
  const int64_t pps = g.npx * g.npy * g.npz;
  for (int64_t p = (int64_t)blockIdx.x * kGbWarps + (threadIdx.x >> 5); p < g.nrec;
       p += (int64_t)gridDim.x * kGbWarps) {
    const int64_t t = p / pps, rem = p - t * pps;
    const int64_t bz = rem / (g.npx * g.npy), r2 = rem - bz * g.npx * g.npy;
    const int64_t by = r2 / g.npx, bx = r2 - by * g.npx;
    const int64_t x0 = bx * g.px, y0 = by * g.py, z0 = bz * g.pz;
    for (int i = lane; i < M; i += 32) {
      const int ix = i % g.px, iy = (i / g.px) % g.py, iz = i / (g.px * g.py);
      W.u[i] = (double)in[((t * g.dims[2] + z0 + iz) * g.dims[1] + (y0 + iy)) * g.dims[0] + (x0 + ix)];
    }
    __syncwarp();
    // alpha = Phi^T u (each a sequential fma sum over the components), q
    for (int k = lane; k < M; k += 32) {
      double a = 0.0;
      for (int j = 0; j < M; ++j) a = __fma_rn(phi[j * M + k], W.u[j], a);
      W.al[k] = a;
      long long q = 0;
      if (delta > 0.0) {
        const double y = rint(__ddiv_rn(a, delta));
        if (!(fabs(y) < 0x1p62)) atomicOr(&st->overflow, 1u);
        else q = (long long)y;
      }
      W.q[k] = q;
      W.qd[k] = __dmul_rn((double)q, delta);
    }
    __syncwarp();
    // ranks by |alpha| (descending, index order on ties) on the magnitudes'
    // bit patterns: for non-negative doubles their order is the integers'
    // order, and the comparisons leave the FP64 pipe to the arithmetic
    for (int k = lane; k < M; k += 32) {
      const unsigned long long ak = (unsigned long long)__double_as_longlong(W.al[k]) & 0x7FFFFFFFFFFFFFFFull;
      int rank = 0;
      for (int j = 0; j < M; ++j) {
        const unsigned long long aj = (unsigned long long)__double_as_longlong(W.al[j]) & 0x7FFFFFFFFFFFFFFFull;
        rank += (aj > ak || (aj == ak && j < k)) ? 1 : 0;
      }
      W.ord[rank] = k;
    }
    __syncwarp();
    // the smallest kept count by bisection over [0, M]
    int n = 0;
    if (delta > 0.0) {
      int lo = 0, hi = M;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        double part = 0.0;
        for (int i = lane; i < M; i += 32) {
          double rec = 0.0;
          for (int s = 0; s < mid; ++s) {
            const int k = W.ord[s];
            rec = __dadd_rn(rec, __dmul_rn(W.qd[k], phi[i * M + k]));
          }
          const double d = __dsub_rn(W.u[i], rec);
          part = __fma_rn(d, d, part);
        }
        if (gb_warp_sum(part) <= eps_l2) hi = mid;
        else lo = mid + 1;
      }
      n = lo;
    }
    // the record: n, wv, n mode indices of ib bits, n zigzag(q) of wv bits
    uint64_t zmax = 0;
    for (int s = lane; s < n; s += 32) {
      const uint64_t z = gb_zz(W.q[W.ord[s]]);
      zmax = z > zmax ? z : zmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t z = __shfl_xor_sync(0xffffffffu, zmax, o);
      zmax = z > zmax ? z : zmax;
    }
    const int wv = gb_width(zmax);
    const int64_t nbits = (int64_t)n * (ib + wv);
    const int nw = (int)((nbits + 31) / 32);
    const int64_t bytes = align_up(8 + 4 * (int64_t)nw, 8);
    for (int w = lane; w < nw + 2; w += 32) W.words[w] = 0u;
    __syncwarp();
    for (int s = lane; s < n; s += 32) {
      const int k = W.ord[s];
      gb_put(W.words, (uint64_t)s * ib, (uint64_t)k, ib);
      gb_put(W.words, (uint64_t)n * ib + (uint64_t)s * wv, gb_zz(W.q[k]), wv);
    }
    __syncwarp();
    uint32_t* slot = reinterpret_cast<uint32_t*>(slots + p * g.slot_bytes);
    for (int w = lane; w < (int)(bytes / 4); w += 32)
      slot[w] = w == 0 ? (uint32_t)n : w == 1 ? (uint32_t)wv : W.words[w - 2];
    if (lane == 0) sizes[p] = (unsigned long long)bytes;
    __syncwarp();
  }
}

// ---------------------------------------------------------------- the stream
// One CTA: the exclusive scan of the record sizes (in place into offsets),
// the total, and the header, basis and offset table when they fit.
__global__ void __launch_bounds__(1024) k_gb_scan(GbPlan g, const unsigned long long* sizes,
                                                  unsigned long long* offsets, const double* phi, GbStatus* st,
                                                  uint8_t* out, unsigned long long out_cap) {
  __shared__ unsigned long long warp_sums[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < g.nrec; base += 1024) {
    const int64_t i = base + tid;
    const unsigned long long v = i < g.nrec ? sizes[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const unsigned long long excl = carry + (warp > 0 ? warp_sums[warp - 1] : 0ull) + x - v;
    if (i < g.nrec) offsets[i] = excl;
    __syncthreads();
    if (tid == 1023) carry = excl + v;
    __syncthreads();
  }
  const unsigned long long payload = carry;
  const unsigned long long total = (unsigned long long)g.payload_pos + payload;
  if (tid == 0) {
    offsets[g.nrec] = payload;
    st->total = total;
  }
  if (total > out_cap) return;
  const int M = g.M;
  if (tid == 0) {
    uint32_t* h32 = reinterpret_cast<uint32_t*>(out);
    uint64_t* h64 = reinterpret_cast<uint64_t*>(out);
    double* hd = reinterpret_cast<double*>(out);
    h32[0] = kGbMagic;
    h32[1] = 1u;
    h32[2] = (uint32_t)M;
    h32[3] = (uint32_t)g.px;
    h32[4] = (uint32_t)g.py;
    h32[5] = (uint32_t)g.pz;
    for (int a = 0; a < 4; ++a) h64[3 + a] = (uint64_t)g.dims[a];
    hd[7] = st->eps_l2;
    hd[8] = st->delta;
    h64[9] = (uint64_t)g.nrec;
  }
  double* basis = reinterpret_cast<double*>(out + kGbHdr);
  for (int e = tid; e < M * M; e += 1024) {
    const int r = e / M, i = e - r * M;          // mode r, component i
    basis[e] = phi[i * M + r];
  }
  uint64_t* ot = reinterpret_cast<uint64_t*>(out + g.offsets_pos);
  for (int64_t i = tid; i <= g.nrec; i += 1024) ot[i] = offsets[i];
}

// The records from their slots to their offsets (8-byte words).
__global__ void k_gb_copy(GbPlan g, const unsigned long long* sizes, const unsigned long long* offsets,
                          const uint8_t* slots, const GbStatus* st, uint8_t* out, unsigned long long out_cap) {
  if (st->total > out_cap) return;
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= g.nrec) return;
  const int lane = threadIdx.x & 31;
  const uint2* src = reinterpret_cast<const uint2*>(slots + p * g.slot_bytes);
  uint2* dst = reinterpret_cast<uint2*>(out + g.payload_pos + offsets[p]);
  for (int64_t w = lane; w < (int64_t)(sizes[p] / 8); w += 32) dst[w] = src[w];
}

// ---------------------------------------------------------------- decoder
// A warp per record: its mode indices and values, then each point the sum of
// (q_s delta) phi_s over the kept modes in kept order.
__global__ void __launch_bounds__(256) k_gb_decode(GbPlan g, const uint8_t* __restrict__ comp,
                                                   unsigned long long comp_bytes, double delta, double* out,
                                                   GbStatus* st) {
  const int64_t p = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= g.nrec) return;
  const int lane = threadIdx.x & 31;
  const int M = g.M;
  const uint64_t* ot = reinterpret_cast<const uint64_t*>(comp + g.offsets_pos);
  const double* basis = reinterpret_cast<const double*>(comp + kGbHdr);   // [mode][component]
  const uint64_t o0 = ot[p], o1 = ot[p + 1];
  if (o1 < o0 + 8 || (uint64_t)g.payload_pos + o1 > comp_bytes || (o0 & 7) != 0) {
    if (lane == 0) atomicOr(&st->corrupt, 1u);
    return;
  }
  const uint32_t* r = reinterpret_cast<const uint32_t*>(comp + g.payload_pos + o0);
  const int n = (int)r[0], wv = (int)(r[1] & 0xFFu);
  const int ib = g.ib;
  if (n > M || wv > 63 || (r[1] >> 8) != 0u ||
      (int64_t)(o1 - o0) != align_up(8 + 4 * (((int64_t)n * (ib + wv) + 31) / 32), 8)) {
    if (lane == 0) atomicOr(&st->corrupt, 1u);
    return;
  }
  const uint32_t* w = r + 2;
  auto get = [&](uint64_t pos, int width) -> uint64_t {
    uint64_t v = 0;
    for (int done = 0; done < width;) {
      const int sh = (int)(pos & 31);
      const int take = (32 - sh) < (width - done) ? (32 - sh) : (width - done);
      const uint64_t part = (w[pos >> 5] >> sh) & ((take == 32) ? 0xFFFFFFFFull : ((1ull << take) - 1ull));
      v |= part << done;
      pos += (uint64_t)take;
      done += take;
    }
    return v;
  };
  const int64_t pps = g.npx * g.npy * g.npz;
  const int64_t t = p / pps, rem = p - t * pps;
  const int64_t bz = rem / (g.npx * g.npy), r2 = rem - bz * g.npx * g.npy;
  const int64_t by = r2 / g.npx, bx = r2 - by * g.npx;
  const int64_t x0 = bx * g.px, y0 = by * g.py, z0 = bz * g.pz;
  for (int i = lane; i < M; i += 32) {
    double rec = 0.0;
    for (int s = 0; s < n; ++s) {
      const int k = (int)get((uint64_t)s * ib, ib);
      const uint64_t z = get((uint64_t)n * ib + (uint64_t)s * wv, wv);
      const long long q = (long long)((z >> 1) ^ (0ull - (z & 1ull)));
      if (k >= M) {
        if (lane == 0) atomicOr(&st->corrupt, 1u);
        return;
      }
      rec = __dadd_rn(rec, __dmul_rn(__dmul_rn((double)q, delta), basis[(int64_t)k * M + i]));
    }
    const int ix = i % g.px, iy = (i / g.px) % g.py, iz = i / (g.px * g.py);
    out[((t * g.dims[2] + z0 + iz) * g.dims[1] + (y0 + iy)) * g.dims[0] + (x0 + ix)] = rec;
  }
}

}  // namespace
}  // namespace dls

using namespace dls;

size_t dls_gb_bound(const dls_gb_params* p) {
  GbPlan g;
  if (gb_make_plan(p, &g) != DLS_OK) return 0;
  return (size_t)(g.payload_pos + g.nrec * gb_record_max(g.M, g.ib));
}

size_t dls_gb_workspace_size(const dls_gb_params* p) {
  GbPlan g;
  if (gb_make_plan(p, &g) != DLS_OK) return 0;
  return gb_layout(g).total;
}

int dls_gb_compress(const dls_gb_params* p, const float* d_in, const int64_t* d_origins, void* d_out, size_t out_cap,
                    size_t* out_bytes, void* d_workspace, size_t ws_bytes, dls_stream_t stream) {
  GbPlan g;
  int st = gb_make_plan(p, &g);
  if (st != DLS_OK) return st;
  if (!d_in || !d_origins || !d_out || !out_bytes || ((uintptr_t)d_out & 15) || ((uintptr_t)d_in & 3) ||
      ((uintptr_t)d_origins & 7))
    return DLS_ERR_INVALID_ARG;
  const GbLayout L = gb_layout(g);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* w = (uint8_t*)d_workspace;
  double* Q = (double*)(w + L.Q);
  double* G = (double*)(w + L.G);
  double* V = (double*)(w + L.V);
  double* phi = (double*)(w + L.phi);
  double* lam = (double*)(w + L.lam);
  double* partial = (double*)(w + L.partial);
  GbStatus* gs = (GbStatus*)(w + L.status);
  unsigned long long* sizes = (unsigned long long*)(w + L.sizes);
  unsigned long long* offsets = (unsigned long long*)(w + L.offsets);
  uint8_t* slots = w + L.slots;
  if (cudaMemsetAsync(gs, 0, sizeof(GbStatus), s) != cudaSuccess) return DLS_ERR_CUDA;
  k_gb_sample<<<(unsigned)g.S, 128, 0, s>>>(g, d_in, d_origins, Q, gs);
  k_gb_gram<<<(unsigned)cdiv((int64_t)g.M * g.M, 256), 256, 0, s>>>(g, Q, G);
  // V beside A in shared memory when both fit (M <= 90), else in global memory
  const int me = g.M + (g.M & 1);
  const int v_shared = 2 * sizeof(double) * (size_t)me * me <= 200 * 1024 ? 1 : 0;
  const size_t jsm = sizeof(double) * (size_t)me * me * (v_shared ? 2 : 1);
  if (cudaFuncSetAttribute(k_gb_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm) != cudaSuccess)
    return DLS_ERR_CUDA;
  k_gb_jacobi<<<1, kJacThreads, jsm, s>>>(g, G, V, phi, lam, v_shared);
  k_gb_norm<<<kGbStatCtas, 256, 0, s>>>(g, d_in, partial, gs);
  k_gb_resolve<<<1, 1, 0, s>>>(g, partial, gs);
  const size_t psm = gb_patch_smem(g.M);
  if (cudaFuncSetAttribute(k_gb_patch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm) != cudaSuccess)
    return DLS_ERR_CUDA;
  int per = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gb_patch, kGbWarps * 32, psm) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DLS_ERR_CUDA;
  if (per < 1) return DLS_ERR_CUDA;
  const int64_t need = cdiv(g.nrec, kGbWarps);
  const unsigned grid = (unsigned)((int64_t)per * sms < need ? (int64_t)per * sms : need);
  k_gb_patch<<<grid, kGbWarps * 32, psm, s>>>(g, d_in, phi, gs, gs, sizes, slots);
  k_gb_scan<<<1, 1024, 0, s>>>(g, sizes, offsets, phi, gs, (uint8_t*)d_out, (unsigned long long)out_cap);
  k_gb_copy<<<(unsigned)cdiv(g.nrec, 8), 256, 0, s>>>(g, sizes, offsets, slots, gs, (uint8_t*)d_out,
                                                     (unsigned long long)out_cap);
  if (cudaGetLastError() != cudaSuccess) return DLS_ERR_CUDA;
  GbStatus hs;
  if (cudaMemcpyAsync(&hs, gs, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DLS_ERR_CUDA;
  if (hs.bad_origin || hs.overflow) return DLS_ERR_INVALID_ARG;
  if (hs.nonfinite) return DLS_ERR_NONFINITE;
  *out_bytes = (size_t)hs.total;
  return hs.total > out_cap ? DLS_ERR_CAPACITY : DLS_OK;
}

int dls_gb_decompress(const void* d_comp, size_t comp_bytes, double* d_out, size_t out_count, dls_stream_t stream) {
  if (!d_comp || !d_out || comp_bytes < (size_t)kGbHdr || ((uintptr_t)d_comp & 15) || ((uintptr_t)d_out & 7))
    return DLS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t h[kGbHdr];
  if (cudaMemcpyAsync(h, d_comp, kGbHdr, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return DLS_ERR_CUDA;
  uint32_t h32[6];
  uint64_t dims[4], nrec;
  double eps_l2, delta;
  memcpy(h32, h, 24);
  memcpy(dims, h + 24, 32);
  memcpy(&eps_l2, h + 56, 8);
  memcpy(&delta, h + 64, 8);
  memcpy(&nrec, h + 72, 8);
  if (h32[0] != kGbMagic || h32[1] != 1u || h32[3] == 0 || h32[3] != h32[4] || h32[2] > (uint32_t)kGbMaxM)
    return DLS_ERR_CORRUPT;
  for (int a = 0; a < 4; ++a)
    if (dims[a] < 1 || dims[a] > (1ull << 40)) return DLS_ERR_CORRUPT;
  dls_gb_params p;
  p.m = (int32_t)h32[3];
  for (int a = 0; a < 4; ++a) p.dims[a] = (int64_t)dims[a];
  p.eps_t = 1.0;
  p.nsample = 1;
  GbPlan g;
  if (gb_make_plan(&p, &g) != DLS_OK || (uint32_t)g.M != h32[2] || (uint32_t)g.pz != h32[5] ||
      (uint64_t)g.nrec != nrec || !isfinite(delta) || delta < 0.0)
    return DLS_ERR_CORRUPT;
  if (comp_bytes < (size_t)g.payload_pos) return DLS_ERR_CORRUPT;
  if (out_count < (size_t)g.K) return DLS_ERR_CAPACITY;
  // the offset table: starts at 0, ends at the stream's end (the records' own
  // sizes are checked on the device)
  uint64_t first = 0, last = 0;
  const uint8_t* c = (const uint8_t*)d_comp;
  if (cudaMemcpyAsync(&first, c + g.offsets_pos, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&last, c + g.offsets_pos + 8 * g.nrec, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DLS_ERR_CUDA;
  if (first != 0 || (uint64_t)g.payload_pos + last != (uint64_t)comp_bytes) return DLS_ERR_CORRUPT;
  GbStatus* gs = nullptr;
  if (cudaMallocAsync((void**)&gs, sizeof(GbStatus), s) != cudaSuccess) return DLS_ERR_CUDA;
  if (cudaMemsetAsync(gs, 0, sizeof(GbStatus), s) != cudaSuccess) {
    cudaFreeAsync(gs, s);
    return DLS_ERR_CUDA;
  }
  if (g.nrec > 0)
    k_gb_decode<<<(unsigned)cdiv(g.nrec, 8), 256, 0, s>>>(g, c, (unsigned long long)comp_bytes, delta, d_out, gs);
  GbStatus hs;
  memset(&hs, 0, sizeof(hs));
  const bool launched = cudaGetLastError() == cudaSuccess;
  cudaMemcpyAsync(&hs, gs, sizeof(hs), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(gs, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || !launched) return DLS_ERR_CUDA;
  return hs.corrupt ? DLS_ERR_CORRUPT : DLS_OK;
}
