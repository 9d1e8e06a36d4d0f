// The lossless stage on the pointwise corrections (Sec. 2.5 and Algorithm 1
// step 3 of arXiv 2601.20113 follow the lossy map with a lossless coder, undone
// first in Sec. 2.6): a record's correction section may be Rice coded (record
// flag 8) where that is strictly smaller than its dense or entry-list form.
//
// The corrections k[0..N) of a block, in element order, escaped points as
// zeros, are cut into chunks of 1024 elements.  In a chunk every nonzero is
// written as the Rice code of the count of zeros before it (from the chunk
// start or the previous nonzero), then zigzag(k) - 1 in wv bits; one more Rice
// code gives the zeros up to the chunk end.  The Rice code of a count c with
// parameter kr is (c >> kr) one bits, a zero bit, then the kr low bits of c.
// Bits run LSB first in 32-bit words, chunk after chunk, and the section is
// [coded words, kr | wv << 8, the chunks' bit offsets, the coded words], so
// that chunks decode independently.  wv is the bit width of the largest
// zigzag(k) - 1; kr in [0, 20] takes the fewest bits (the smallest on ties).
//
// The stage runs after the record packers, on the stream they wrote into a
// staging buffer: k_rice_plan sizes every record's Rice section and decides,
// the scan writes the final header and offsets, and k_rice_write copies each
// record to its final place, coding the section where it was chosen.  A warp
// takes a chunk, each lane 32 consecutive elements of it; the run before a
// lane's first nonzero comes from a max-scan of the lanes' last nonzero
// positions, and a lane's first code bit from a scan of the lanes' code
// lengths.  The counts per record come from one pass over its corrections:
// sum over runs of (run >> kr) = sum_i c_i 2^(i - kr) over the bits i >= kr,
// with c_i the number of runs whose bit i is set, so every kr is priced from
// eleven counters (a run is at most 1024).
#include "dls_device.cuh"

namespace dls {
namespace {

constexpr int kRiceThreads = 256;
constexpr int kRunBits = 11;               // runs are <= kRiceChunk = 2^10

__device__ __forceinline__ uint32_t rd_bits(const uint32_t* w, uint64_t pos, int width) {
  if (width == 0) return 0u;
  const uint64_t wi = pos >> 5;
  const int sh = (int)(pos & 31);
  uint64_t v = (uint64_t)w[wi] >> sh;
  if (sh + width > 32) v |= (uint64_t)w[wi + 1] << (32 - sh);
  return width >= 32 ? (uint32_t)v : (uint32_t)v & ((1u << width) - 1u);
}

// A packed record's correction section, as the packers wrote it.
struct CorrSrc {
  const uint32_t* cw;
  int wk, ib, dense;
  int64_t ncorr, nesc;
  RecLayout lay;
};

// Parses the record at `rec` (written by this library's packers); false for a
// raw record or one without corrections.
__device__ bool corr_src(const Geom& g, const uint8_t* rec, int es, CorrSrc& s) {
  const uint32_t* rec32 = reinterpret_cast<const uint32_t*>(rec);
  const int r = rec[0], flags = rec[1];
  if (flags & kFlagRaw) return false;
  s.wk = rec[2];
  s.ib = rec[3];
  s.ncorr = rec32[1];
  s.nesc = rec32[2];
  if (s.wk == 0) return false;
  s.lay = rec_layout(r, g.n, g.L, g.N, es, rec + 16, s.wk, s.ib, s.ncorr, s.nesc);
  s.dense = s.lay.dense;
  s.cw = reinterpret_cast<const uint32_t*>(rec + s.lay.off_c);
  return true;
}


// A warp's view of one chunk in shared memory: mask[L] holds the nonzeros of
// elements c0 + 32 L .. c0 + 32 L + 31 (lane L's part), z[33 L + i] the
// zigzag value of element c0 + 32 L + i where its bit is set (escapes are
// zeros in both source forms).
struct WarpChunk {
  uint32_t mask[32];
  uint32_t z[32 * 33];
};

// Lane L's 32 dense fields of width WK (compile time): WK words from p, of
// which the first cnt fields are the chunk's.
template <int WK>
__device__ __forceinline__ uint32_t dense_fields(const uint32_t* p, int cnt, uint32_t* z) {
  uint32_t w[WK];
  const int nw = (cnt * WK + 31) >> 5;
#pragma unroll
  for (int k = 0; k < WK; ++k) w[k] = k < nw ? p[k] : 0u;
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    constexpr uint32_t fm = (1u << WK) - 1u;
    const int b = i * WK, k = b >> 5, sh = b & 31;
    uint32_t f = w[k] >> sh;
    if (sh + WK > 32) f |= w[k + 1] << (32 - sh);
    f &= fm;
    if (i < cnt && f != 0u) {
      m |= 1u << i;
      z[i] = f;
    }
  }
  return m;
}

// Fills the warp's view of chunk [c0, c1) (all lanes of the warp); an
// entry-list source's entries of the chunk are [lo, hi).
__device__ void load_chunk(const CorrSrc& s, int64_t c0, int64_t c1, int64_t lo, int64_t hi, int lane,
                           WarpChunk& V) {
  if (s.dense && s.wk <= 8) {
    const int64_t e0 = c0 + 32 * (int64_t)lane;
    const int cnt = e0 >= c1 ? 0 : (int)((c1 - e0) < 32 ? (c1 - e0) : 32);
    const uint32_t* p = s.cw + (e0 >> 5) * s.wk;
    uint32_t* z = V.z + 33 * lane;
    uint32_t m = 0;
    switch (s.wk) {
      case 1: m = dense_fields<1>(p, cnt, z); break;
      case 2: m = dense_fields<2>(p, cnt, z); break;
      case 3: m = dense_fields<3>(p, cnt, z); break;
      case 4: m = dense_fields<4>(p, cnt, z); break;
      case 5: m = dense_fields<5>(p, cnt, z); break;
      case 6: m = dense_fields<6>(p, cnt, z); break;
      case 7: m = dense_fields<7>(p, cnt, z); break;
      default: m = dense_fields<8>(p, cnt, z); break;
    }
    V.mask[lane] = m;
    __syncwarp();
    return;
  }
  if (s.dense) {
    // lane L's 32 fields start at bit (c0 + 32 L) wk: a word boundary
    const int64_t e0 = c0 + 32 * (int64_t)lane;
    const int cnt = e0 >= c1 ? 0 : (int)((c1 - e0) < 32 ? (c1 - e0) : 32);
    const int wk = s.wk;
    const uint64_t fm = wk >= 32 ? 0xFFFFFFFFull : ((1ull << wk) - 1ull);
    const uint32_t* p = s.cw + (e0 >> 5) * wk;
    uint64_t buf = 0;
    int nb = 0;
    uint32_t m = 0;
    for (int i = 0; i < cnt; ++i) {
      if (nb < wk) {
        buf |= (uint64_t)(*p++) << nb;
        nb += 32;
      }
      const uint32_t z = (uint32_t)(buf & fm);
      buf >>= wk;
      nb -= wk;
      if (z != 0u) {
        m |= 1u << i;
        V.z[33 * lane + i] = z;
      }
    }
    V.mask[lane] = m;
    __syncwarp();
    return;
  }
  V.mask[lane] = 0u;
  __syncwarp();
  const int W = s.ib + s.wk;
  for (int64_t j = lo + lane; j < hi; j += 32) {
    const uint64_t pos = (uint64_t)j * W;
    const int d = (int)((int64_t)rd_bits(s.cw, pos, s.ib) - c0);
    if (d < 0 || d >= kRiceChunk) continue;     // entries are the chunk's (the packers sort them)
    atomicOr(&V.mask[d >> 5], 1u << (d & 31));
    V.z[33 * (d >> 5) + (d & 31)] = rd_bits(s.cw, pos + s.ib, s.wk);
  }
  __syncwarp();
}

// Entry-list sources: every chunk's first entry into chunks[c].first (all
// threads of the CTA; entries in increasing element order).
__device__ void chunk_firsts(const CorrSrc& s, int64_t nch, RiceChunk* chunks) {
  const int W = s.ib + s.wk;
  if (s.ncorr == 0)
    for (int64_t c = threadIdx.x; c < nch; c += blockDim.x) chunks[c].first = 0u;
  for (int64_t j = threadIdx.x; j < s.ncorr; j += blockDim.x) {
    const int64_t cj = (int64_t)rd_bits(s.cw, (uint64_t)j * W, s.ib) / kRiceChunk;
    const int64_t cp = j > 0 ? (int64_t)rd_bits(s.cw, (uint64_t)(j - 1) * W, s.ib) / kRiceChunk : -1;
    for (int64_t c = cp + 1; c <= cj && c < nch; ++c) chunks[c].first = (uint32_t)j;
    if (j == s.ncorr - 1)
      for (int64_t c = cj + 1; c < nch; ++c) chunks[c].first = (uint32_t)s.ncorr;
  }
}

__device__ __forceinline__ void chunk_entries(const CorrSrc& s, const RiceChunk* chunks, int64_t ch, int64_t nch,
                                              int64_t* lo, int64_t* hi) {
  if (s.dense) {
    *lo = *hi = 0;
    return;
  }
  *lo = chunks[ch].first;
  *hi = ch + 1 < nch ? (int64_t)chunks[ch + 1].first : s.ncorr;
  if (*hi > s.ncorr) *hi = s.ncorr;              // within the record's entry list
  if (*lo > *hi) *lo = *hi;
}

// A lane's part of chunk [c0, c1): its first and last nonzero (-1 when none)
// and, through a warp max-scan, the last nonzero before it and the chunk's
// last nonzero (c0 - 1 when none).
struct LaneView {
  int64_t e0;
  uint32_t m;
  int32_t first, last, prev, chunk_last;
};

__device__ __forceinline__ LaneView lane_view(const WarpChunk& V, int64_t c0, int lane) {
  LaneView v;
  v.e0 = c0 + 32 * (int64_t)lane;
  v.m = V.mask[lane];
  v.first = v.m ? (int32_t)(v.e0 + __ffs(v.m) - 1) : -1;
  v.last = v.m ? (int32_t)(v.e0 + 31 - __clz(v.m)) : -1;
  int32_t incl = v.last >= 0 ? v.last : (int32_t)(c0 - 1);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = t > incl ? t : incl;
  }
  const int32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
  v.prev = lane == 0 ? (int32_t)(c0 - 1) : ex;
  v.chunk_last = __shfl_sync(0xffffffffu, incl, 31);
  return v;
}

// f(run, e, z) for the lane's nonzeros in element order, run = the zeros
// before each (from the previous nonzero, or the lane view's prev).
template <class F>
__device__ __forceinline__ void lane_codes(const WarpChunk& V, const LaneView& v, int lane, F f) {
  int64_t prev = v.prev;
  for (uint32_t mm = v.m; mm; mm &= mm - 1) {
    const int i = __ffs(mm) - 1;
    const int64_t e = v.e0 + i;
    f((uint64_t)(e - prev - 1), e, V.z[33 * lane + i]);
    prev = e;
  }
}

// Code bits of a lane's part with parameters (kr, wv): its nonzeros' codes
// and, in the last lane, the chunk's closing code.
__device__ __forceinline__ uint32_t lane_bits(const WarpChunk& V, const LaneView& v, int64_t c1, int lane, int kr,
                                              int wv) {
  uint32_t bits = 0;
  lane_codes(V, v, lane, [&](uint64_t run, int64_t, uint32_t) {
    bits += ((uint32_t)run >> kr) + 1u + (uint32_t)kr + (uint32_t)wv;
  });
  if (lane == 31) bits += ((uint32_t)(c1 - 1 - v.chunk_last) >> kr) + 1u + (uint32_t)kr;
  return bits;
}

__device__ __forceinline__ uint32_t warp_excl_sum(uint32_t x, int lane, uint32_t* total) {
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  *total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - x;
}

// Writer of one chunk's bits from bit `pos` on: whole words inside the chunk
// are stored, the first and the last (which the neighbouring chunks may
// share) are OR-ed into words zeroed beforehand.
// Words at or past `limit` are not written (the sizes disagreed: `over` is set).
struct BitEmit {
  uint32_t* w;
  uint64_t word, limit;
  uint64_t acc;
  int fill;
  bool first, over;
  __device__ BitEmit(uint32_t* words, uint64_t pos, uint64_t nwords)
      : w(words), word(pos >> 5), limit(nwords), acc(0), fill((int)(pos & 31)), first(true), over(false) {}
  __device__ __forceinline__ void put(uint32_t v, int width) {   // v < 2^width, width <= 32
    if (width == 0) return;
    acc |= (uint64_t)v << fill;
    fill += width;
    if (fill >= 32) {
      if (word >= limit) over = true;
      else if (first) atomicOr(&w[word], (uint32_t)acc);
      else w[word] = (uint32_t)acc;
      first = false;
      ++word;
      acc >>= 32;
      fill -= 32;
    }
  }
  __device__ void ones(uint64_t u) {
    for (; u >= 32; u -= 32) put(0xFFFFFFFFu, 32);
    if (u) put((1u << u) - 1u, (int)u);
  }
  __device__ void code(uint64_t run, int kr) {
    ones(run >> kr);
    put(0u, 1);
    put((uint32_t)(run & ((1ull << kr) - 1ull)), kr);
  }
  __device__ void finish() {
    if (fill > 0 && acc != 0) {
      if (word >= limit) over = true;
      else atomicOr(&w[word], (uint32_t)acc);
    }
  }
};

__device__ __forceinline__ const uint8_t* src_record(const Plan& P, const uint8_t* s0, int64_t bi, int64_t* bytes) {
  const uint64_t* offs = reinterpret_cast<const uint64_t*>(s0 + P.offsets_pos);
  *bytes = (int64_t)(offs[bi + 1] - offs[bi]);
  return s0 + P.payload_pos + offs[bi];
}

// One CTA per record: the run statistics, the parameters, and the choice
// (Rice where 2 + chunks + coded words is strictly below the current section);
// a chosen record's new size goes to meta[bi].nbytes for the scan.
__global__ void __launch_bounds__(kRiceThreads) k_rice_plan(Plan P, const uint8_t* __restrict__ s0,
                                                           BlockMeta* meta, RiceInfo* info, RiceChunk* chunks,
                                                           const Status* st) {
  __shared__ unsigned long long cnt[kRunBits + 1];          // bit counts of the runs, then nonzeros
  __shared__ unsigned int vor_sh;
  __shared__ WarpChunk views[kRiceThreads / 32];
  const int64_t bi = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (st->capacity || st->nonfinite || st->timeout) return;
  const int es = P.dtype == DLS_F32 ? 4 : 8;
  const Geom g = block_geom(P, P.b0 + bi);
  int64_t bytes;
  const uint8_t* rec = src_record(P, s0, bi, &bytes);
  CorrSrc src;
  if (!corr_src(g, rec, es, src)) {
    if (tid == 0) info[bi] = RiceInfo{0u, 0, 0, 0};
    return;
  }
  if (tid <= kRunBits) cnt[tid] = 0ull;
  if (tid == 0) vor_sh = 0u;
  __syncthreads();
  const int64_t N = g.N, nch = cdiv(N, kRiceChunk);
  uint32_t c[kRunBits];
#pragma unroll
  for (int i = 0; i < kRunBits; ++i) c[i] = 0u;
  uint32_t nz = 0u, vor = 0u;
  auto count = [&](uint32_t run) {
#pragma unroll
    for (int i = 0; i < kRunBits; ++i) c[i] += (run >> i) & 1u;
  };
  WarpChunk& V = views[warp];
  RiceChunk* rc = chunks + bi * rice_chunks_per_block(P);
  if (!src.dense) {
    chunk_firsts(src, nch, rc);
    __syncthreads();
  }
  uint32_t wsum[kRunBits + 1];                       // lane 0: this warp's totals
#pragma unroll
  for (int i = 0; i <= kRunBits; ++i) wsum[i] = 0u;
  for (int64_t ch = warp; ch < nch; ch += kRiceThreads / 32) {
    const int64_t c0 = ch * kRiceChunk, c1 = (c0 + kRiceChunk) < N ? c0 + kRiceChunk : N;
    int64_t lo, hi;
    chunk_entries(src, rc, ch, nch, &lo, &hi);
    load_chunk(src, c0, c1, lo, hi, lane, V);
    const LaneView v = lane_view(V, c0, lane);
#pragma unroll
    for (int i = 0; i < kRunBits; ++i) c[i] = 0u;
    nz = 0u;
    lane_codes(V, v, lane, [&](uint64_t run, int64_t, uint32_t z) {
      count((uint32_t)run);
      ++nz;
      vor |= z - 1u;
    });
    if (lane == 31) count((uint32_t)(c1 - 1 - v.chunk_last));
    // the chunk's counts (runs <= 1025, so 16 bits each)
    RiceChunk rec_c;
#pragma unroll
    for (int i = 0; i <= kRunBits; ++i) {
      const uint32_t x = __reduce_add_sync(0xffffffffu, i < kRunBits ? c[i] : nz);
      if (i < kRunBits) rec_c.c[i] = (uint16_t)x;
      else rec_c.nnz = (uint16_t)x;
      wsum[i] += x;
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kRunBits; ++i) rc[ch].c[i] = rec_c.c[i];
      rc[ch].nnz = rec_c.nnz;
    }
    __syncwarp();
  }
  {
    const uint32_t y = __reduce_or_sync(0xffffffffu, vor);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i <= kRunBits; ++i)
        if (wsum[i]) atomicAdd(&cnt[i], (unsigned long long)wsum[i]);
      atomicOr(&vor_sh, y);
    }
  }
  __syncthreads();
  if (tid != 0) return;
  const int wv = bit_width(vor_sh);
  const uint64_t nnz = cnt[kRunBits], nruns = nnz + (uint64_t)nch;
  uint64_t best = 0;
  int bkr = 0;
  for (int kr = 0; kr <= kRiceMaxKr; ++kr) {
    uint64_t sum = 0;
    for (int i = kr; i < kRunBits; ++i) sum += cnt[i] << (i - kr);
    const uint64_t bits = sum + nruns * (uint64_t)(1 + kr) + nnz * (uint64_t)wv;
    if (kr == 0 || bits < best) {
      best = bits;
      bkr = kr;
    }
  }
  const int64_t words = (int64_t)((best + 31) / 32);
  if (2 + nch + words < src.lay.corr_words) {
    const RecLayout nl = rice_layout(src.lay, N, words, src.nesc, es);
    meta[bi].nbytes = nl.size;
    info[bi] = RiceInfo{(uint32_t)words, bkr, wv, 1};
  } else {
    meta[bi].nbytes = bytes;
    info[bi] = RiceInfo{0u, 0, 0, 0};
  }
}

// One CTA per record: the record at its final offset, with the Rice section
// where k_rice_plan chose it (zeroed first, so padding stays zero).
__global__ void __launch_bounds__(kRiceThreads) k_rice_write(Plan P, const uint8_t* __restrict__ s0,
                                                            const unsigned long long* __restrict__ new_off,
                                                            const RiceInfo* __restrict__ info,
                                                            const RiceChunk* __restrict__ chunks, uint8_t* out,
                                                            Status* st_w) {
  __shared__ int sh_warp[32];
  __shared__ WarpChunk views[kRiceThreads / 32];
  const Status* st = st_w;
  const int64_t bi = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (st->capacity || st->nonfinite || st->timeout) return;
  const int es = P.dtype == DLS_F32 ? 4 : 8;
  int64_t bytes;
  const uint8_t* rec = src_record(P, s0, bi, &bytes);
  uint8_t* dst = out + P.payload_pos + new_off[bi];
  const RiceInfo ri = info[bi];
  if (!ri.on) {
    const uint4* a = reinterpret_cast<const uint4*>(rec);
    uint4* b = reinterpret_cast<uint4*>(dst);
    for (int64_t i = tid; i < bytes / 16; i += kRiceThreads) b[i] = a[i];
    return;
  }
  const Geom g = block_geom(P, P.b0 + bi);
  CorrSrc src;
  corr_src(g, rec, es, src);
  const int64_t N = g.N, nch = cdiv(N, kRiceChunk);
  const int kr = ri.kr, wv = ri.wv;
  const RecLayout nl = rice_layout(src.lay, N, ri.words, src.nesc, es);
  for (int64_t i = tid; i < nl.size / 16; i += kRiceThreads) reinterpret_cast<uint4*>(dst)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  // the prefix up to the corrections (8-byte multiple), then the escapes
  for (int64_t i = tid; i < nl.off_c / 8; i += kRiceThreads)
    reinterpret_cast<uint2*>(dst)[i] = reinterpret_cast<const uint2*>(rec)[i];
  for (int64_t i = tid; i < src.nesc; i += kRiceThreads)
    reinterpret_cast<uint32_t*>(dst + nl.off_ei)[i] = reinterpret_cast<const uint32_t*>(rec + src.lay.off_ei)[i];
  for (int64_t i = tid; i < src.nesc * es / 4; i += kRiceThreads)
    reinterpret_cast<uint32_t*>(dst + nl.off_ev)[i] = reinterpret_cast<const uint32_t*>(rec + src.lay.off_ev)[i];
  uint32_t* cw = reinterpret_cast<uint32_t*>(dst + nl.off_c);
  uint32_t* tab = cw + 2;
  uint32_t* words = cw + 2 + nch;
  // chunk sizes in bits, then their exclusive scan in place
  WarpChunk& V = views[warp];
  const RiceChunk* rc = chunks + bi * rice_chunks_per_block(P);
  for (int64_t ch = tid; ch < nch; ch += kRiceThreads) {
    // the chunk's code length: its runs' (run >> kr), a zero and kr bits per
    // run (nonzeros + the closing run), wv bits per nonzero
    const RiceChunk c = rc[ch];
    uint32_t sum = 0;
    for (int i = kr; i < kRunBits; ++i) sum += (uint32_t)c.c[i] << (i - kr);
    tab[ch] = sum + ((uint32_t)c.nnz + 1u) * (uint32_t)(1 + kr) + (uint32_t)c.nnz * (uint32_t)wv;
  }
  __syncthreads();
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nch; b0 += kRiceThreads) {
    const int64_t i = b0 + tid;
    const int x = i < nch ? (int)tab[i] : 0;
    int tot;
    const int ex = block_excl_scan(x, sh_warp, &tot);
    if (i < nch) tab[i] = carry + (uint32_t)ex;
    carry += (uint32_t)tot;
  }
  if (tid == 0) {
    dst[1] = (uint8_t)((rec[1] & ~kFlagDense) | kFlagRice);
    reinterpret_cast<uint32_t*>(dst)[3] = (uint32_t)nl.size;
    cw[0] = ri.words;
    cw[1] = (uint32_t)kr | ((uint32_t)wv << 8);
  }
  __syncthreads();
  // the codes: each lane from its own first bit
  for (int64_t ch = warp; ch < nch; ch += kRiceThreads / 32) {
    const int64_t c0 = ch * kRiceChunk, c1 = (c0 + kRiceChunk) < N ? c0 + kRiceChunk : N;
    int64_t lo, hi;
    chunk_entries(src, rc, ch, nch, &lo, &hi);
    load_chunk(src, c0, c1, lo, hi, lane, V);
    const LaneView v = lane_view(V, c0, lane);
    uint32_t tot;
    const uint32_t off = warp_excl_sum(lane_bits(V, v, c1, lane, kr, wv), lane, &tot);
    BitEmit em(words, (uint64_t)tab[ch] + off, ri.words);
    lane_codes(V, v, lane, [&](uint64_t run, int64_t, uint32_t z) {
      em.code(run, kr);
      em.put(z - 1u, wv);
    });
    if (lane == 31) em.code((uint64_t)(c1 - 1 - v.chunk_last), kr);
    em.finish();
    if (em.over) atomicOr(&st_w->corrupt, 1u);
    __syncwarp();
  }
}

}  // namespace

// The stage over a stream the packers wrote to `s0` (header, offsets and
// records of the same plan): sizes and choices, the final header and offsets
// into d_out (capacity out_cap), then the records.
int launch_rice(const Plan& p, const Work& w, const uint8_t* s0, RiceInfo* info, RiceChunk* chunks, size_t out_cap,
                void* d_out, cudaStream_t s) {
  if (p.nb > 0) k_rice_plan<<<(unsigned)p.nb, kRiceThreads, 0, s>>>(p, s0, w.meta, info, chunks, w.status);
  int st = launch_scan(p, w, out_cap, d_out, s);
  if (st != DLS_OK) return st;
  if (p.nb > 0)
    k_rice_write<<<(unsigned)p.nb, kRiceThreads, 0, s>>>(p, s0, w.offsets, info, chunks, (uint8_t*)d_out, w.status);
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

}  // namespace dls
