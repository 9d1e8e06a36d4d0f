// Decompression (Sec. 2.6 and Algorithm 2 of arXiv 2601.20113) and
// verification (Sec. 2.4 metrics).
//
// Decode contract: for every point, acc = 0; for k = 0..r-1,
// acc = fma(chat[l][k], Vst[j][k], acc) in the field dtype, with
// chat = dtype(q) * dtype(delta).  Then xtilde = fma(dtype(k), dtype(2eb), acc)
// where the correction k is nonzero, and escaped points take their raw value.
// One CTA per block; every structural field of a record is validated against
// the geometry before use.
#include "dls_internal.cuh"

namespace dls {
namespace {

constexpr int kDecThreads = 256;
// Shared-memory words for a record's coefficient and correction sections
// (72 KB: three CTAs per SM, as the launch bounds ask of the registers).
constexpr int kDecStageWords = 18432;
// Resident CTAs asked of the registers: 3 (80 registers) or 2 (128, no
// spills; faster where records are small, the unrolled rows dominating).
constexpr int kDecMinBlocks = 3;
constexpr int kDecSmallRecord = 32768;     // mean record bytes up to which the 2-CTA form runs

template <typename T> __device__ __forceinline__ T dq(int32_t q, T d);
template <> __device__ __forceinline__ float dq<float>(int32_t q, float d) { return __fmul_rn(__int2float_rn(q), d); }
template <> __device__ __forceinline__ double dq<double>(int32_t q, double d) { return __dmul_rn((double)q, d); }
template <typename T> __device__ __forceinline__ T tf(T a, T b, T c);
template <> __device__ __forceinline__ float tf<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double tf<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ float from_d<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }

__device__ __forceinline__ uint32_t get_bits(const uint32_t* w, uint64_t pos, int width) {
  if (width == 0) return 0;
  const uint64_t wi = pos >> 5;
  const int sh = (int)(pos & 31);
  uint64_t v = w[wi] >> sh;
  if (sh + width > 32) v |= (uint64_t)w[wi + 1] << (32 - sh);
  return (uint32_t)(v & (width == 32 ? 0xffffffffull : ((1ull << width) - 1)));
}

// get_bits for bit positions below 2^32 (a column of L <= 2^26 values of at
// most 32 bits); width 0 reads nothing.
__device__ __forceinline__ uint32_t get_bits32(const uint32_t* w, uint32_t pos, int width) {
  if (width == 0) return 0;
  const uint32_t wi = pos >> 5;
  const int sh = (int)(pos & 31);
  uint32_t v = w[wi] >> sh;
  if (sh + width > 32) v |= w[wi + 1] << (32 - sh);
  return width == 32 ? v : (v & ((1u << width) - 1u));
}

template <int V> struct RankC { static constexpr int value = V; };
template <bool V> struct BoolC { static constexpr bool value = V; };

// Field offset of a block's spatial point ls (x fastest) without the time
// step: 32-bit division (a block's extents are small), once per point.
__device__ __forceinline__ int64_t spatial_off(const Plan& p, const Geom& g, int ls) {
  const int sx = g.sx, sxy = g.sx * g.sy;
  const int lz = ls / sxy, rxy = ls - lz * sxy;
  const int ly = rxy / sx, lx = rxy - ly * sx;
  return (int64_t)g.v * p.K + (g.z0 + lz) * (p.dims[0] * p.dims[1]) + (g.y0 + ly) * p.dims[0] + (g.x0 + lx);
}
// elem_index (block element e = t_local * M + s_local) the same way.
__device__ __forceinline__ int64_t elem_off(const Plan& p, const Geom& g, int64_t e) {
  const int64_t lt = e / g.M;
  return spatial_off(p, g, (int)(e - lt * g.M)) + (g.t0 + lt) * p.P;
}

template <typename T, int NM, int MINB>
__global__ void __launch_bounds__(kDecThreads, MINB) k_decode(Plan P, const uint8_t* __restrict__ comp,
                                                        unsigned long long comp_bytes, T* __restrict__ out,
                                                        Status* st) {
  extern __shared__ __align__(16) uint32_t stage_sm[];   // kDecStageWords
  __shared__ T vst[NM * NM];
  __shared__ int64_t wbase[NM + 1];
  __shared__ int64_t soff_col[NM];   // spatial-side blocks: field offset of column j (time 0)
  __shared__ int bad;
  const int64_t bi = blockIdx.x;
  const int tid = threadIdx.x;
  const Geom g = block_geom(P, P.b0 + bi);
  const int64_t N = g.N, L = g.L;
  const int n = g.n;
  const int es = (int)sizeof(T);
  const uint64_t* offs = reinterpret_cast<const uint64_t*>(comp + P.offsets_pos);
  const uint64_t o0 = offs[bi], o1 = offs[bi + 1];
  if (o1 < o0 + 16 || (uint64_t)P.payload_pos + o1 > comp_bytes || (o0 & 15) != 0) {
    if (tid == 0) atomicOr(&st->corrupt, 1u);
    return;
  }
  const uint8_t* rec = comp + P.payload_pos + o0;
  const uint32_t* rec32 = reinterpret_cast<const uint32_t*>(rec);
  const int r = rec[0], flags = rec[1], wk = rec[2], ib = rec[3];
  const int64_t ncorr = rec32[1], nesc = rec32[2], nbytes = rec32[3];
  // a flag outside raw / spatial side / dense / Rice-coded corrections is refused
  if (nbytes != (int64_t)(o1 - o0) || nbytes < 16 ||
      (flags & ~(int)(kFlagRaw | kFlagSpatial | kFlagDense | kFlagRice)) != 0) {
    if (tid == 0) atomicOr(&st->corrupt, 1u);
    return;
  }
  if (flags & kFlagRaw) {
    if (16 + N * es > nbytes) {
      if (tid == 0) atomicOr(&st->corrupt, 1u);
      return;
    }
    const T* vals = reinterpret_cast<const T*>(rec + 16);
    for (int64_t e = tid; e < N; e += kDecThreads) out[elem_off(P, g, e)] = vals[e];
    return;
  }
  const int rcap = P.rank_cap < n ? P.rank_cap : n;
  const uint8_t* wq = rec + 16;
  if (tid == 0) {
    bad = 0;
    if (16 + align_up(r, 8) > nbytes || r > rcap || wk > 32 || ib != bit_width((uint32_t)(N - 1)) || ncorr > N || nesc > N ||
        (((flags & kFlagSpatial) ? 1 : 0) != g.side))
      bad = 1;
    int64_t acc = 0;
    for (int c = 0; c < r && !bad; ++c) {
      if (wq[c] > 32) bad = 1;
      wbase[c] = acc;
      acc += (L * wq[c] + 31) / 32;
    }
    wbase[r] = acc;
    if (!bad) {
      RecLayout lay = rec_layout(r, n, L, N, es, wq, wk, ib, ncorr, nesc);
      if (flags & kFlagRice) {
        // [coded words, kr | wv << 8, chunk bit offsets, coded words]
        if (wk == 0 || (flags & kFlagDense) || lay.off_c + 8 > nbytes) {
          bad = 1;
        } else {
          const uint32_t* cw = reinterpret_cast<const uint32_t*>(rec + lay.off_c);
          if ((cw[1] >> 16) != 0u || (int)(cw[1] & 0xFFu) > kRiceMaxKr || (int)((cw[1] >> 8) & 0xFFu) > 32 ||
              (int64_t)cw[0] > nbytes)
            bad = 1;
          else
            lay = rice_layout(lay, N, cw[0], nesc, es);
        }
        if (!bad && lay.size != nbytes) bad = 1;
      } else if (lay.size != nbytes || (lay.dense ? 1 : 0) != ((flags & kFlagDense) ? 1 : 0)) {
        bad = 1;
      }
    }
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicOr(&st->corrupt, 1u);
    return;
  }
  const bool rice = (flags & kFlagRice) != 0;
  RecLayout lay = rec_layout(r, n, L, N, es, wq, wk, ib, ncorr, nesc);
  if (rice) lay = rice_layout(lay, N, reinterpret_cast<const uint32_t*>(rec + lay.off_c)[0], nesc, es);
  const int v = g.v;
  const double delta = reinterpret_cast<const double*>(comp + kHdr + kVarRec * v)[2];
  const double step = reinterpret_cast<const double*>(comp + kHdr + kVarRec * v)[3];
  const T delta_t = from_d<T>(delta), step_t = from_d<T>(step);
  const T* vin = reinterpret_cast<const T*>(rec + lay.off_v);
  for (int i = tid; i < n * r; i += kDecThreads) {
    const int c = i / n, j = i - c * n;
    vst[j * NM + c] = vin[i];
  }
  if (g.side == 1 && tid < n) soff_col[tid] = spatial_off(P, g, tid);
  // the coefficient and correction sections (contiguous words from off_q) go
  // to shared memory in one pass with every load in flight, when they fit;
  // the row loop then reads them at shared-memory latency
  const int64_t cw_at = (lay.off_c - lay.off_q) / 4;
  const int64_t nstage = cw_at + lay.corr_words;
  const bool staged = nstage <= kDecStageWords;
  const uint32_t* qw = reinterpret_cast<const uint32_t*>(rec + lay.off_q);
  if (staged)
    for (int64_t i = tid; i < nstage; i += kDecThreads) stage_sm[i] = qw[i];
  __syncthreads();
  if (staged) qw = stage_sm;
  const uint32_t* cw = qw + cw_at;
  const bool dense = lay.dense && wk > 0;
  // Rank 1-8 (the common case) with the rank fixed at compile time: the
  // coefficients of a row in registers, each output r FMAs; the time-side
  // outputs of a row one time plane apart.  Other ranks: guarded up to NM.
  auto rows_fixed = [&](auto RK) {
    constexpr int R = decltype(RK)::value;
    int wqc[R];
    const uint32_t* qc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) { wqc[c] = wq[c]; qc[c] = qw + wbase[c]; }
    for (int64_t l = tid; l < L; l += kDecThreads) {
      const int64_t row_off = g.side == 0 ? spatial_off(P, g, (int)l) + g.t0 * P.P : (g.t0 + l) * P.P;
      T ch[R];
#pragma unroll
      for (int c = 0; c < R; ++c) ch[c] = dq<T>(unzigzag(get_bits32(qc[c], (uint32_t)l * (uint32_t)wqc[c], wqc[c])), delta_t);
      T* o = out + row_off;
#pragma unroll 1
      for (int j = 0; j < n; ++j) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < R; ++c) acc = tf<T>(ch[c], vst[j * NM + c], acc);
        if (dense) {
          const int32_t kv = unzigzag(get_bits(cw, (uint64_t)a_elem(g, l, j) * wk, wk));
          if (kv != 0) acc = tf<T>((T)kv, step_t, acc);
        }
        if (g.side == 0) {
          *o = acc;
          o += P.P;
        } else {
          out[row_off + soff_col[j]] = acc;
        }
      }
    }
  };
  // Time-side blocks of order 16 (the full 16^3 x 16 blocks) at ranks 1-4: the
  // 16 outputs of a row unrolled, dense corrections read with 32-bit bit
  // positions one time plane (M wk bits) apart (N wk < 2^32 here), blocks
  // without dense corrections compiled without their test.
  auto rows_t16 = [&](auto RK, auto DK) {
    constexpr int R = decltype(RK)::value;
    constexpr bool D = decltype(DK)::value;
    int wqc[R];
    const uint32_t* qc[R];
#pragma unroll
    for (int c = 0; c < R; ++c) { wqc[c] = wq[c]; qc[c] = qw + wbase[c]; }
    const uint32_t pstep = (uint32_t)g.M * (uint32_t)wk;
    for (int l = tid; l < (int)L; l += kDecThreads) {
      T ch[R];
#pragma unroll
      for (int c = 0; c < R; ++c) ch[c] = dq<T>(unzigzag(get_bits32(qc[c], (uint32_t)l * (uint32_t)wqc[c], wqc[c])), delta_t);
      T* o = out + spatial_off(P, g, l) + g.t0 * P.P;
      uint32_t pos = (uint32_t)l * (uint32_t)wk;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < R; ++c) acc = tf<T>(ch[c], vst[j * NM + c], acc);
        if (D) {
          const int32_t kv = unzigzag(get_bits32(cw, pos, wk));
          pos += pstep;
          if (kv != 0) acc = tf<T>((T)kv, step_t, acc);
        }
        *o = acc;
        o += P.P;
      }
    }
  };
  auto rows_t16_d = [&](auto RK) {
    if (dense) rows_t16(RK, BoolC<true>());
    else rows_t16(RK, BoolC<false>());
  };
  if (NM == 16 && g.side == 0 && n == 16 && r >= 1 && r <= 4) {
    switch (r) {
      case 1: rows_t16_d(RankC<1>()); break;
      case 2: rows_t16_d(RankC<2>()); break;
      case 3: rows_t16_d(RankC<3>()); break;
      default: rows_t16_d(RankC<4>()); break;
    }
  } else switch (r) {
    case 1: rows_fixed(RankC<1>()); break;
    case 2: rows_fixed(RankC<2>()); break;
    case 3: rows_fixed(RankC<3>()); break;
    case 4: rows_fixed(RankC<4>()); break;
    case 5: rows_fixed(RankC<5>()); break;
    case 6: rows_fixed(RankC<6>()); break;
    case 7: rows_fixed(RankC<7>()); break;
    case 8: rows_fixed(RankC<8>()); break;
    default:
      for (int64_t l = tid; l < L; l += kDecThreads) {
        // row l's field offset: a spatial point (time side) or a time step (spatial side)
        const int64_t row_off = g.side == 0 ? spatial_off(P, g, (int)l) + g.t0 * P.P : (g.t0 + l) * P.P;
        T ch[NM];
#pragma unroll
        for (int c = 0; c < NM; ++c) {
          if (c < r) {
            const uint32_t z = get_bits(qw + wbase[c], (uint64_t)l * wq[c], wq[c]);
            ch[c] = dq<T>(unzigzag(z), delta_t);
          } else {
            ch[c] = T(0);
          }
        }
        // one output at a time: unrolled over j, the basis (loop-invariant over
        // rows) would be held in registers, a CTA per SM
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
          {
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < NM; ++c)
              if (c < r) acc = tf<T>(ch[c], vst[j * NM + c], acc);
            const int64_t e = a_elem(g, l, j);
            if (dense) {
              const int32_t kv = unzigzag(get_bits(cw, (uint64_t)e * wk, wk));
              if (kv != 0) acc = tf<T>((T)kv, step_t, acc);
            }
            out[row_off + (g.side == 0 ? (int64_t)j * P.P : soff_col[j])] = acc;
          }
        }
      }
      break;
  }
  __syncthreads();
  if (rice) {
    // chunk by chunk, one thread each: a Rice code gives the zeros before
    // the next nonzero (or the chunk's end), then wv bits give zigzag(k) - 1
    const int kr = (int)(cw[1] & 0xFFu), wv = (int)((cw[1] >> 8) & 0xFFu);
    const int64_t nch = cdiv(N, kRiceChunk);
    const uint32_t* rw = cw + 2 + nch;
    const uint64_t nbits = (uint64_t)cw[0] * 32;
    for (int64_t ch = tid; ch < nch; ch += kDecThreads) {
      const int64_t c1 = (ch + 1) * kRiceChunk < N ? (ch + 1) * kRiceChunk : N;
      int64_t e = ch * kRiceChunk;
      uint64_t pos = cw[2 + ch];
      bool ok = true;
      int64_t pg[8];
      int32_t pk[8];
      int npend = 0;
      auto flush = [&]() {
        T val[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) val[b] = b < npend ? out[pg[b]] : T(0);
#pragma unroll
        for (int b = 0; b < 8; ++b)
          if (b < npend) out[pg[b]] = tf<T>((T)pk[b], step_t, val[b]);
        npend = 0;
      };
      for (;;) {
        // the unary part: ones up to a zero
        uint64_t q = 0;
        for (;;) {
          if (pos >= nbits) { ok = false; break; }
          const int avail = (nbits - pos) < 32 ? (int)(nbits - pos) : 32;
          const uint32_t w = get_bits(rw, pos, avail);
          const int t = (~w == 0u) ? 32 : __ffs(~w) - 1;
          if (t >= avail) {
            q += (uint64_t)avail;
            pos += (uint64_t)avail;
            if (q > (uint64_t)kRiceChunk) { ok = false; break; }
            continue;
          }
          q += (uint64_t)t;
          pos += (uint64_t)t + 1;
          break;
        }
        if (!ok || pos + (uint64_t)kr > nbits) { ok = false; break; }
        const uint64_t run = (q << kr) | get_bits(rw, pos, kr);
        pos += (uint64_t)kr;
        if (run > (uint64_t)(c1 - e)) { ok = false; break; }
        e += (int64_t)run;
        if (e == c1) break;
        if (pos + (uint64_t)wv > nbits) { ok = false; break; }
        const int32_t kv = unzigzag(get_bits(rw, pos, wv) + 1u);
        pos += (uint64_t)wv;
        // the read-backs of the outputs go eight at a time (distinct elements)
        pg[npend] = elem_off(P, g, e);
        pk[npend] = kv;
        if (++npend == 8) flush();
        ++e;
      }
      flush();
      if (!ok) atomicOr(&st->corrupt, 1u);
    }
  } else if (!dense && wk > 0) {
    // entry-list corrections read the rows' outputs back: eight entries a
    // thread at a time, all eight loads issued before the first store, so that
    // the read-backs overlap (entries name distinct elements)
    constexpr int kB = 8;
    for (int64_t i0 = tid; i0 < ncorr; i0 += (int64_t)kB * kDecThreads) {
      int64_t gi[kB];
      int32_t kv[kB];
      T val[kB];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int64_t i = i0 + (int64_t)b * kDecThreads;
        gi[b] = -1;
        kv[b] = 0;
        if (i < ncorr) {
          const uint64_t pos = (uint64_t)i * (uint64_t)(ib + wk);
          const int64_t e = get_bits(cw, pos, ib);
          kv[b] = unzigzag(get_bits(cw, pos + ib, wk));
          if (e >= N) atomicOr(&st->corrupt, 1u);
          else gi[b] = elem_off(P, g, e);
        }
      }
#pragma unroll
      for (int b = 0; b < kB; ++b) val[b] = gi[b] >= 0 ? out[gi[b]] : T(0);
#pragma unroll
      for (int b = 0; b < kB; ++b)
        if (gi[b] >= 0) out[gi[b]] = tf<T>((T)kv[b], step_t, val[b]);
    }
  }
  __syncthreads();
  if (nesc > 0) {
    const uint32_t* ei = reinterpret_cast<const uint32_t*>(rec + lay.off_ei);
    const T* ev = reinterpret_cast<const T*>(rec + lay.off_ev);
    for (int64_t i = tid; i < nesc; i += kDecThreads) {
      const int64_t e = ei[i];
      if (e >= N) { atomicOr(&st->corrupt, 1u); continue; }
      out[elem_off(P, g, e)] = ev[i];
    }
  }
}

// ---------------------------------------------------------------- verification
// acc layout (doubles): per variable v (16 doubles): [0] max_abs_err key (as
// u64), [1] n_over (u64), [2] sum_sq_err, [3] sum_sq; then stream totals at
// 16*nvars: [0] n_raw, [1] sum rank, [2] n_corr, [3] n_esc, [4] basis bytes,
// [5] coeff bytes, [6] corr bytes, [7] esc bytes, [8] raw bytes, [9] header bytes.
template <typename T>
__global__ void __launch_bounds__(256) k_verify_points(Plan P, const T* __restrict__ a, const T* __restrict__ b,
                                                       const uint8_t* comp, double* acc) {
  const int v = blockIdx.y;
  const double eb = reinterpret_cast<const double*>(comp + kHdr + kVarRec * v)[1];
  const bool pointwise = P.eb_type != DLS_EB_NRMSE;
  double mx = 0.0, se = 0.0, sx = 0.0;
  unsigned long long over = 0;
  const int64_t base = (int64_t)v * P.K;
  for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < P.K; i += (int64_t)gridDim.x * 256) {
    const double x = (double)a[base + i], y = (double)b[base + i];
    const double d = fabs(x - y);
    mx = fmax(mx, d);
    if (pointwise && d > eb) ++over;
    se = fma(d, d, se);
    sx = fma(x, x, sx);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    over += __shfl_xor_sync(0xffffffffu, over, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* u = reinterpret_cast<unsigned long long*>(acc + 16 * v);
    atomicMax(&u[0], dkey(mx));
    atomicAdd(&u[1], over);
    atomicAdd(&acc[16 * v + 2], se);
    atomicAdd(&acc[16 * v + 3], sx);
  }
}

// float32 fields: the same report with the FP64 pipe kept for what needs it.
// A point's difference is s = fl32(x - y) and its rounding error e (TwoSum,
// s + e = x - y exactly); the bound test decides in FP32 outside a relative
// 2^-20 band around eb and in FP64 inside it; the maximum is taken in FP64 on
// the points whose |s| reaches the thread's running maximum (rounding is
// monotone, so the point of the largest |x - y| is among them); the sums of
// squares run as unevaluated float pairs (x^2 = p + fma(x, x, -p) exactly,
// d^2 = s^2 + 2 s e to within e^2 <= 2^-48 s^2) per batch of 1024 points of a
// thread, each batch then added in FP64.  Values beyond 2^60 take the FP64
// path.  Loads are float4 when the field allows (4 | K, 16-byte pointers).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float a, float ae) {
  const float s = __fadd_rn(hi, a);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, ae));
}

// The FP64 work of a point, out of line so that it runs only when taken
// (inlined, it would be predicated and issued for every point).
__device__ __noinline__ double fp64_diff(float x, float y) { return fabs((double)x - (double)y); }

__global__ void __launch_bounds__(256) k_verify_points_f32(Plan P, const float* __restrict__ a,
                                                           const float* __restrict__ b, const uint8_t* comp,
                                                           double* acc, int vec4) {
  const int v = blockIdx.y;
  const double eb = reinterpret_cast<const double*>(comp + kHdr + kVarRec * v)[1];
  const bool pointwise = P.eb_type != DLS_EB_NRMSE;
  const float eb_lo = __double2float_rd(eb * (1.0 - 0x1p-20)), eb_hi = __double2float_ru(eb * (1.0 + 0x1p-20));
  const float big = 0x1p60f;
  double mx = 0.0, se = 0.0, sx = 0.0;
  float mx32 = 0.0f;
  unsigned long long over = 0;
  float eh = 0.0f, el = 0.0f, xh = 0.0f, xl = 0.0f;
  auto point = [&](float x, float y) {
    const float sd = __fsub_rn(x, y);
    const float bb = __fsub_rn(sd, x);
    const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(sd, bb)), __fsub_rn(-y, bb));
    const float ad = fabsf(sd);
    if (!(fabsf(x) < big) || !(fabsf(y) < big) || !(ad < big)) {
      // far out of range (or not finite): this point in FP64
      const double d = fp64_diff(x, y);
      mx = fmax(mx, d);
      if (pointwise && d > eb) ++over;
      se = fma(d, d, se);
      sx = fma((double)x, (double)x, sx);
      return;
    }
    if (ad >= mx32 && ad > 0.0f) {
      mx32 = ad;
      mx = fmax(mx, fp64_diff(x, y));
    }
    if (pointwise) {
      if (ad > eb_hi) ++over;
      else if (ad >= eb_lo && fp64_diff(x, y) > eb) ++over;
    }
    const float p = __fmul_rn(sd, sd);
    ff_add(eh, el, p, __fmaf_rn(__fmul_rn(2.0f, sd), e, __fmaf_rn(sd, sd, -p)));
    const float q = __fmul_rn(x, x);
    ff_add(xh, xl, q, __fmaf_rn(x, x, -q));
  };
  auto flush = [&]() {
    se += (double)eh + (double)el;
    sx += (double)xh + (double)xl;
    eh = el = xh = xl = 0.0f;
  };
  const int64_t base = (int64_t)v * P.K;
  const int64_t stride = (int64_t)gridDim.x * 256;
  if (vec4) {
    // four points a load; batches of 256 loads (1024 points) per float pair
    const float4* a4 = reinterpret_cast<const float4*>(a + base);
    const float4* b4 = reinterpret_cast<const float4*>(b + base);
    const int64_t K4 = P.K / 4;
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    while (i < K4) {
#pragma unroll 4
      for (int n = 0; n < 256 && i < K4; ++n, i += stride) {
        const float4 x = a4[i], y = b4[i];
        point(x.x, y.x);
        point(x.y, y.y);
        point(x.z, y.z);
        point(x.w, y.w);
      }
      flush();
    }
  } else {
    int64_t i = blockIdx.x * 256ll + threadIdx.x;
    while (i < P.K) {
      for (int n = 0; n < 1024 && i < P.K; ++n, i += stride) point(a[base + i], b[base + i]);
      flush();
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    over += __shfl_xor_sync(0xffffffffu, over, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* u = reinterpret_cast<unsigned long long*>(acc + 16 * v);
    atomicMax(&u[0], dkey(mx));
    atomicAdd(&u[1], over);
    atomicAdd(&acc[16 * v + 2], se);
    atomicAdd(&acc[16 * v + 3], sx);
  }
}

__global__ void k_verify_stream(Plan P, const uint8_t* comp, unsigned long long comp_bytes, int es, double* acc) {
  const int64_t bi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (bi >= P.nb) return;
  const Geom g = block_geom(P, P.b0 + bi);
  const uint64_t* offs = reinterpret_cast<const uint64_t*>(comp + P.offsets_pos);
  const uint64_t o0 = offs[bi], o1 = offs[bi + 1];
  if (o1 < o0 + 16 || (uint64_t)P.payload_pos + o1 > comp_bytes || (o0 & 15) != 0) return;
  const uint8_t* rec = comp + P.payload_pos + o0;
  const uint32_t* rec32 = reinterpret_cast<const uint32_t*>(rec);
  double* t = acc + 16 * P.nvars;
  const int r = rec[0], flags = rec[1];
  if (!(flags & kFlagRaw) && (r > kMaxN || 16 + align_up(r, 8) > (int64_t)(o1 - o0))) return;
  if (flags & kFlagRaw) {
    atomicAdd(&t[0], 1.0);
    atomicAdd(&t[8], (double)rec32[3]);
    return;
  }
  RecLayout lay = rec_layout(r, g.n, g.L, g.N, es, rec + 16, rec[2], rec[3], rec32[1], rec32[2]);
  if ((flags & kFlagRice) && lay.off_c + 4 <= (int64_t)(o1 - o0))
    lay = rice_layout(lay, g.N, reinterpret_cast<const uint32_t*>(rec + lay.off_c)[0], rec32[2], es);
  atomicAdd(&t[1], (double)r);
  atomicAdd(&t[2], (double)rec32[1]);
  atomicAdd(&t[3], (double)rec32[2]);
  atomicAdd(&t[4], (double)(lay.off_q - lay.off_v));
  atomicAdd(&t[5], (double)(lay.off_c - lay.off_q));
  atomicAdd(&t[6], (double)(lay.off_ei - lay.off_c));
  atomicAdd(&t[7], (double)(lay.size - lay.off_ei));
  atomicAdd(&t[9], (double)lay.off_v);
}

}  // namespace

int launch_decode(const Plan& p, const void* d_comp, unsigned long long comp_bytes, void* d_out,
                        Status* st, cudaStream_t s) {
  if (p.nb == 0) return DLS_OK;
  const unsigned grid = (unsigned)p.nb;
  const uint8_t* c = (const uint8_t*)d_comp;
  const int sm = kDecStageWords * 4;
  // the stage buffer is above the 48 KB default: opt in before each launch
  auto go = [&](auto kern, auto* outp) -> bool {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return false;
    kern<<<grid, kDecThreads, sm, s>>>(p, c, comp_bytes, outp, st);
    return true;
  };
  bool ok;
  // measured on 16^3 x 16 float32 blocks: 2 CTAs per SM 1.78 ms against 2.13 at
  // 1e-3 (21 KB records), 3 CTAs 3.52 against 3.79 at 1e-4 (52 KB records)
  const bool small = comp_bytes / (unsigned long long)p.nb <= (unsigned long long)kDecSmallRecord;
  if (p.dtype == DLS_F32) {
    if (p.nmax <= 16)
      ok = small ? go(k_decode<float, 16, 2>, (float*)d_out) : go(k_decode<float, 16, kDecMinBlocks>, (float*)d_out);
    else
      ok = go(k_decode<float, 32, kDecMinBlocks>, (float*)d_out);
  } else {
    ok = p.nmax <= 16 ? go(k_decode<double, 16, kDecMinBlocks>, (double*)d_out)
                      : go(k_decode<double, 32, kDecMinBlocks>, (double*)d_out);
  }
  return ok && cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

int launch_verify(const Plan& p, const void* d_orig, const void* d_recon, const void* d_comp,
                  unsigned long long comp_bytes, double* acc, cudaStream_t s) {
  dim3 grid(1024, p.nvars);
  if (p.dtype == DLS_F32)
    k_verify_points_f32<<<grid, 256, 0, s>>>(p, (const float*)d_orig, (const float*)d_recon, (const uint8_t*)d_comp, acc,
                                             (p.K % 4 == 0 && ((uintptr_t)d_orig & 15) == 0 &&
                                              ((uintptr_t)d_recon & 15) == 0) ? 1 : 0);
  else
    k_verify_points<double><<<grid, 256, 0, s>>>(p, (const double*)d_orig, (const double*)d_recon, (const uint8_t*)d_comp, acc);
  if (p.nb > 0)
    k_verify_stream<<<(unsigned)cdiv(p.nb, 256), 256, 0, s>>>(p, (const uint8_t*)d_comp, comp_bytes, p.dtype == DLS_F32 ? 4 : 8, acc);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

}  // namespace dls
