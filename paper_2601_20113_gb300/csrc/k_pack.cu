// Stream assembly: exclusive scan of record sizes (the GPU form of the
// paper's MPI_Scan for write positions, Sec. 2.7.2), the addressable header
// and offset table, and the per-block record packer.
//
// Record layout (all offsets relative to the 16-byte aligned record start):
//   [0,16)  u8 r, u8 flags, u8 w_k, u8 ib, u32 n_corr, u32 n_esc, u32 nbytes
//   w_q[r] bytes, padded to 8
//   Vst: for k < r, for j < n: Vst[j][k] in the field dtype, padded to 8
//   q: for k < r: ceil(L*w_q[k]/32) u32 words of zigzag(q[l][k]), LSB first
//   corrections: dense  -> zigzag(k[e]) for every element e at w_k bits
//                sparse -> per nonzero k (increasing e): e (ib bits), zigzag(k) (w_k bits)
//   escapes: n_esc u32 element indices, padded to 8; n_esc raw values, padded to 8
//   record padded to 16.  Raw record: header with RAW flag + N values in element order.
#include "dls_device.cuh"

namespace dls {
namespace {

constexpr int kPackThreads = 256;

// ---------------------------------------------------------------- scan + header
__global__ void __launch_bounds__(1024) k_scan_header(Plan P, Work W, uint8_t* out, unsigned long long out_cap) {
  __shared__ unsigned long long warp_sums[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (W.status->nonfinite) return;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < P.nb; base += 1024) {
    const int64_t i = base + tid;
    unsigned long long v = (i < P.nb) ? (unsigned long long)W.meta[i].nbytes : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const unsigned long long excl = carry + (warp > 0 ? warp_sums[warp - 1] : 0ull) + x - v;
    if (i < P.nb) W.offsets[i] = excl;
    __syncthreads();
    if (tid == 1023) carry = excl + v;
    __syncthreads();
  }
  const unsigned long long total_payload = carry;
  const unsigned long long total = (unsigned long long)P.payload_pos + total_payload;
  if (tid == 0) {
    W.offsets[P.nb] = total_payload;
    W.status->total_bytes = total;
    if (total > out_cap) W.status->capacity = 1u;
  }
  if (total > out_cap) return;
  // header, variable table, offset table
  uint8_t* o = out;
  for (int64_t i = tid; i < P.payload_pos; i += 1024) o[i] = 0;
  __syncthreads();
  if (tid == 0) {
    uint32_t* o32 = (uint32_t*)o;
    uint64_t* o64 = (uint64_t*)o;
    o32[0] = kMagic;
    o32[1] = kVersion;
    o32[2] = kHdr;
    o32[3] = (uint32_t)P.nvars;
    for (int a = 0; a < 4; ++a) o64[2 + a] = (uint64_t)P.dims[a];
    for (int a = 0; a < 4; ++a) o32[12 + a] = (uint32_t)P.block[a];
    o[64] = (uint8_t)P.dtype;
    o[65] = (uint8_t)P.eb_type;
    o[66] = (uint8_t)P.precision;
    o[67] = (uint8_t)P.rank_mode;
    o32[17] = (uint32_t)P.rank_cap;
    o64[9] = (uint64_t)P.b0;
    o64[10] = (uint64_t)(P.b0 + P.nb);
    o64[11] = (uint64_t)P.nb_total;
    o64[12] = (uint64_t)kHdr;
    o64[13] = (uint64_t)P.offsets_pos;
    o64[14] = (uint64_t)P.payload_pos;
    o64[15] = (uint64_t)total;
  }
  for (int v = tid; v < P.nvars; v += 1024) {
    double* vr = (double*)(o + kHdr + kVarRec * v);
    vr[0] = W.vars[v].eb_user;
    vr[1] = W.vars[v].eb;
    vr[2] = W.vars[v].delta;
    vr[3] = W.vars[v].step;
  }
  uint64_t* offt = (uint64_t*)(o + P.offsets_pos);
  for (int64_t i = tid; i <= P.nb; i += 1024) offt[i] = W.offsets[i];
}

template <typename T>
__global__ void __launch_bounds__(kPackThreads) k_pack(Plan P, const T* __restrict__ in, Work W, uint8_t* out) {
  if (W.status->capacity || W.status->nonfinite) return;
  __shared__ int sh_warp[32];
  __shared__ BlockMeta m;
  const int64_t bi = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) m = W.meta[bi];
  __syncthreads();
  const Geom g = block_geom(P, P.b0 + bi);
  const int64_t N = g.N, L = g.L;
  const int n = g.n;
  const int es = (int)sizeof(T);
  uint8_t* rec = out + P.payload_pos + W.offsets[bi];
  // zero the record
  for (int64_t i = tid; i < m.nbytes / 16; i += kPackThreads) reinterpret_cast<uint4*>(rec)[i] = make_uint4(0, 0, 0, 0);
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
    T* vals = reinterpret_cast<T*>(rec + 16);
    for (int64_t e = tid; e < N; e += kPackThreads) {
      const int64_t lt = e / g.M, ls = e - lt * g.M;
      vals[e] = in[elem_index(P, g, ls, lt)];
    }
    return;
  }
  const int r = m.r;
  const RecLayout lay = rec_layout(r, n, L, N, es, m.wq, m.wk, m.ib, m.ncorr, m.nesc);
  for (int c = tid; c < r; c += kPackThreads) rec[lay.off_wq + c] = m.wq[c];
  const double* vst = W.vst + bi * (int64_t)P.nmax * P.nmax;
  const int rcap = m.rcap;
  T* vout = reinterpret_cast<T*>(rec + lay.off_v);
  for (int i = tid; i < n * r; i += kPackThreads) {
    const int c = i / n, j = i - c * n;
    vout[i] = (T)vst[j * rcap + c];
  }
  // coefficient columns
  const int32_t* qb = W.q + (g.pt_off - P.pt_base);
  uint32_t* qw = reinterpret_cast<uint32_t*>(rec + lay.off_q);
  int64_t wbase = 0;
  for (int c = 0; c < r; ++c) {
    const int wdt = m.wq[c];
    const int64_t words = (L * wdt + 31) / 32;
    const int32_t* col = qb + (int64_t)c * L;
    for (int64_t w = tid; w < words; w += kPackThreads)
      qw[wbase + w] = compose_word(w, wdt, L, [&](int64_t l) { return zigzag(col[l]); });
    wbase += words;
  }
  // corrections
  const int32_t* kb = W.kc + (g.pt_off - P.pt_base);
  uint32_t* cw = reinterpret_cast<uint32_t*>(rec + lay.off_c);
  if (m.wk > 0) {
    if (lay.dense) {
      for (int64_t w = tid; w < lay.corr_words; w += kPackThreads)
        cw[w] = compose_word(w, m.wk, N, [&](int64_t e) {
          const int32_t kv = kb[e];
          return kv == kEscape ? 0u : zigzag(kv);
        });
    } else {
      int base = 0;
      for (int64_t e0 = 0; e0 < N; e0 += kPackThreads) {
        const int64_t e = e0 + tid;
        const int32_t kv = e < N ? kb[e] : 0;
        const int flag = (e < N && kv != 0 && kv != kEscape) ? 1 : 0;
        int tot;
        const int ex = block_excl_scan(flag, sh_warp, &tot);
        if (flag) {
          const uint64_t pos = (uint64_t)(base + ex) * (uint64_t)(m.ib + m.wk);
          or_bits(cw, pos, (uint32_t)e, m.ib);
          or_bits(cw, pos + m.ib, zigzag(kv), m.wk);
        }
        base += tot;
      }
    }
  }
  // escapes
  if (m.nesc > 0) {
    uint32_t* ei = reinterpret_cast<uint32_t*>(rec + lay.off_ei);
    T* ev = reinterpret_cast<T*>(rec + lay.off_ev);
    int base = 0;
    for (int64_t e0 = 0; e0 < N; e0 += kPackThreads) {
      const int64_t e = e0 + tid;
      const int flag = (e < N && kb[e] == kEscape) ? 1 : 0;
      int tot;
      const int ex = block_excl_scan(flag, sh_warp, &tot);
      if (flag) {
        ei[base + ex] = (uint32_t)e;
        const int64_t lt = e / g.M, ls = e - lt * g.M;
        ev[base + ex] = in[elem_index(P, g, ls, lt)];
      }
      base += tot;
    }
  }
}

// ---------------------------------------------------------------- bound resolution
constexpr int kStatCtas = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_stats(Plan P, const T* __restrict__ in, Work W, double* partial) {
  // grid: (kStatCtas, nvars).  CTA c of variable v reduces a fixed contiguous
  // range in a fixed order, so results are run-to-run deterministic.
  const int v = blockIdx.y, c = blockIdx.x, tid = threadIdx.x;
  const int64_t per = cdiv(P.K, kStatCtas);
  const int64_t i0 = (int64_t)c * per, i1 = min(P.K, i0 + per);
  const T* x = in + (int64_t)v * P.K;
  double s = 0.0;
  double mn = INFINITY, mx = -INFINITY;
  int bad = 0;
  for (int64_t i = i0 + tid; i < i1; i += 256) {
    const double xv = (double)x[i];
    if (!isfinite(xv)) bad = 1;
    s = __fma_rn(xv, xv, s);
    mn = fmin(mn, xv);
    mx = fmax(mx, xv);
  }
  __shared__ double ss[256];
  ss[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) ss[tid] = __dadd_rn(ss[tid], ss[tid + o]);
    __syncthreads();
  }
  if (tid == 0) partial[(int64_t)v * kStatCtas + c] = ss[0];
  if (bad) atomicOr(&W.status->nonfinite, 1u);
  if (mn <= mx) {
    atomicMin(&W.vars[v].minkey, dkey(mn));
    atomicMax(&W.vars[v].maxkey, dkey(mx));
  }
}

// A variable's sum of squares: the CTAs' partial sums added in CTA order.
__device__ double stats_sumsq(const double* partial, int v) {
  double s2 = 0.0;
  for (int c = 0; c < kStatCtas; ++c) s2 = __dadd_rn(s2, partial[(int64_t)v * kStatCtas + c]);
  return s2;
}

__global__ void k_resolve(Plan P, Work W, const double* partial, int have_stats) {
  const int v = threadIdx.x + blockIdx.x * blockDim.x;
  if (v >= P.nvars) return;
  VarInfo& o = W.vars[v];
  const double ebu = P.eb_user[v];
  o.eb_user = ebu;
  double s2 = 0.0;
  double vmin = 0.0, vmax = 0.0;
  if (W.gstats) {
    // the whole field's statistics, given by the caller of a part of it
    vmin = W.gstats[4 * v + 0];
    vmax = W.gstats[4 * v + 1];
    s2 = W.gstats[4 * v + 2];
  } else if (have_stats) {
    s2 = stats_sumsq(partial, v);
    vmin = dunkey(o.minkey);
    vmax = dunkey(o.maxkey);
  }
  o.sumsq = s2;
  if (P.eb_type == DLS_EB_ABS) {
    o.eb = ebu;
  } else if (P.eb_type == DLS_EB_REL_RANGE) {
    const double range = __dsub_rn(vmax, vmin);
    o.eb = range > 0.0 ? __dmul_rn(ebu, range) : ebu;
  } else {
    o.eb = __ddiv_rn(__dmul_rn(ebu, __dsqrt_rn(s2)), 100.0);
  }
  if (P.eb_type == DLS_EB_NRMSE) {
    o.delta = o.eb > 0.0 ? __ddiv_rn(o.eb, __dsqrt_rn(P.kbound)) : 1.0;
    o.step = 0.0;
  } else {
    o.delta = o.eb;
    o.step = __dmul_rn(2.0, o.eb);
  }
}

// The part's own statistics, per variable {min, max, sum of squares, points}.
__global__ void k_stats_export(Plan P, Work W, const double* partial, double* out) {
  const int v = threadIdx.x;
  if (v >= P.nvars) return;
  const VarInfo& o = W.vars[v];
  out[4 * v + 0] = dunkey(o.minkey);
  out[4 * v + 1] = dunkey(o.maxkey);
  out[4 * v + 2] = stats_sumsq(partial, v);
  out[4 * v + 3] = (double)P.K;
}

__global__ void k_init_vars(Plan P, Work W) {
  const int v = threadIdx.x;
  if (v < P.nvars) {
    W.vars[v].minkey = ~0ull;
    W.vars[v].maxkey = 0ull;
  }
}

}  // namespace

int launch_scan(const Plan& p, const Work& w, size_t out_cap, void* d_out, cudaStream_t s) {
  k_scan_header<<<1, 1024, 0, s>>>(p, w, (uint8_t*)d_out, (unsigned long long)out_cap);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_pack(const Plan& p, const void* d_in, const Work& w, void* d_out, size_t, cudaStream_t s) {
  if (p.nb == 0) return DLS_OK;
  if (p.dtype == DLS_F32) k_pack<float><<<(unsigned)p.nb, kPackThreads, 0, s>>>(p, (const float*)d_in, w, (uint8_t*)d_out);
  else k_pack<double><<<(unsigned)p.nb, kPackThreads, 0, s>>>(p, (const double*)d_in, w, (uint8_t*)d_out);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

// Statistics pass (only REL_RANGE / NRMSE need it) followed by resolution.
// `partial` scratch: nvars * kStatCtas doubles, carved from the workspace by the caller.
int launch_stats_resolve(const Plan& p, const void* d_in, const Work& w, double* partial, cudaStream_t s) {
  const bool need = p.eb_type != DLS_EB_ABS && !w.gstats;
  if (need) {
    k_init_vars<<<1, 64, 0, s>>>(p, w);
    dim3 grid(kStatCtas, p.nvars);
    if (p.dtype == DLS_F32) k_stats<float><<<grid, 256, 0, s>>>(p, (const float*)d_in, w, partial);
    else k_stats<double><<<grid, 256, 0, s>>>(p, (const double*)d_in, w, partial);
  }
  k_resolve<<<1, 64, 0, s>>>(p, w, partial, need ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

// The statistics pass alone, its result (nvars x 4 doubles, written to the
// last 4 * nvars doubles of `partial`) copied to h_stats on `s`.
int launch_field_stats(const Plan& p, const void* d_in, const Work& w, double* partial, double* h_stats,
                       cudaStream_t s) {
  double* d_stats = partial + (int64_t)p.nvars * kStatCtas;
  k_init_vars<<<1, 64, 0, s>>>(p, w);
  dim3 grid(kStatCtas, p.nvars);
  if (p.dtype == DLS_F32) k_stats<float><<<grid, 256, 0, s>>>(p, (const float*)d_in, w, partial);
  else k_stats<double><<<grid, 256, 0, s>>>(p, (const double*)d_in, w, partial);
  k_stats_export<<<1, 64, 0, s>>>(p, w, partial, d_stats);
  if (cudaGetLastError() != cudaSuccess) return DLS_ERR_CUDA;
  return cudaMemcpyAsync(h_stats, d_stats, sizeof(double) * 4 * (size_t)p.nvars, cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess
             ? DLS_OK
             : DLS_ERR_CUDA;
}

// CTA partial sums of squares, then the field_stats output (4 per variable).
int stats_partial_doubles(const Plan& p) { return p.nvars * kStatCtas + 4 * p.nvars; }

}  // namespace dls
