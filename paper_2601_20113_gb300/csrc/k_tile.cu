// Staged-tile mixed-precision kernel for float32 fields: the blocks whose
// Gram side is time (T_b <= M_b, Gram order n = T_b <= 16), which is every
// block of the usual shapes.  (Blocks with M_b < T_b go to k_mixed.cu.)
//
// Per block (Algorithm 1 step 3 of arXiv 2601.20113, pointwise-bound reading),
// one CTA of 4 warps, several CTAs per SM, persistent over an atomic counter:
//   Gram pass    the block streams through a two-stage shared-memory ring
//                (TMA tensor tiles, or cp.async where the field's x extent is
//                not 16-byte aligned); FP32 Gram G = A^T A (Sec. 2.7.1) and
//                the block statistics
//   eigensolve   register Jacobi in FP32 (one warp), one FP64 Ogita-Aishima
//                refinement, and a Rayleigh-Ritz pass for tight bounds
//   rank         predicted rank checked exactly, else the bisection of
//                Algorithm 1 on E(r)
//   encode pass  projection, quantization, decode, E(r-1), E(r), pointwise
//                correction, one row per thread from the staged tile
//   pack         the record, written into the block's staging slot with
//                word-aligned bit packing and warp-level compaction
// Every stored decision has FP64 semantics (see mixed_common.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mixed_common.cuh"

namespace dls {
namespace {

constexpr int kTT = 128;                  // threads per CTA
constexpr int kWarps = kTT / 32;
constexpr int kStages = 2;
constexpr int kStageFloats = 4096;        // 16 KiB per stage
constexpr int kNP = NM * (NM + 1) / 2;    // packed Gram pairs (136)
constexpr int kHalf = kNP / 2;            // pairs per thread group (68)
constexpr int kBitsSmem = 8 * NM * NM;    // bitmap words kept in shared memory (2048)
constexpr int kGT = kTT / 2;              // threads per Gram group
constexpr unsigned FULL = 0xffffffffu;
// Bound of every wait on an mbarrier, in SM clock cycles (about a second):
// a poll can return at once, so a bound in polls would be far shorter.
constexpr long long kWaitCycles = 1ll << 31;

enum { kPhGram = 0, kPhJacobi, kPhRefine, kPhRR, kPhPredict, kPhEncode, kPhDecide, kPhSearch, kPhPack,
       kCntAccepted, kCntSearched, kCntExact, kPhTileWait, kCntTcGram, kPhases };
static_assert(kPhases == kMixedPhases, "phase counter layout");

struct TileArgs {
  Plan P;
  const float* in;
  uint8_t* staging;
  BlockMeta* meta;
  VarInfo* vars;
  Status* status;
  int32_t* q_scr;
  int8_t* k8_scr;
  int32_t* k32_scr;
  uint32_t* bit_scr;       // per CTA: nptmax / 32 words
  float* feat;
  int32_t* ranks;
  int64_t lmax, nptmax;
  int learned;
  unsigned long long* phase;
  const MlpModel* model;
  int use_tma;
  int bxb, yc, zc, bt;     // chunk box (x, y, z, t)
  int rc;                  // rows per chunk = bxb * yc * zc
  uint32_t mbx, myc;       // ceil(2^32 / bxb), ceil(2^32 / yc) (0 for a divisor of 1)
  uint32_t mrc;            // ceil(2^32 / rc) (0 for rc = 1)
  int cp_pairs;            // cp.async path: copy x-pairs of 8 bytes (even field and block widths)
  int tc_gram;             // Gram pass on the tensor cores (chunk box 16 x 16 x 1 x 16): a TcMode, 0 for none
  double jfloor;           // Jacobi skip floor as a fraction of the per-mode budget
  int64_t blo, bhi;        // the blocks [blo, bhi) of the plan this launch compresses
  int64_t withhold;        // test hook: the first chunk of this block is never copied (-1: none)
  struct FastBlock* fb;    // per-block state of the phase kernels (plan-relative index)
  struct FastCtl* ctl;     // their block counters and the list k_enc fills
  int32_t* list;           // blocks left to k_tile
  int from_list;           // k_tile: blocks from the list
  int ctas;                // phase-counter slots
};

// Quantization constants of one variable (delta, and 1 / delta and delta in FP32).
struct RowConst {
  double delta;
  float inv_delta, delta_f;
};

// The staging ring is the last member, so that the kernels that stream no
// block (k_eig) allocate only the part before it.
struct __align__(1024) TileSmem {
  unsigned long long full[kStages];
  float G32[NM * NM];
  float Vj[NM * NM];
  float red[kWarps][kNP + 8];
  __align__(16) float VstT[NM * NM];     // VstT[k * NM + j] = Vst[j][k]
  float vsum[NM];
  // FP64 eigen scratch; from the encode pass through the record it holds the
  // nonzero-correction bitmap of blocks of up to kBitsSmem * 32 points
  union {
    struct {
      double G64[NM * NM], X64[NM * NM], R64[NM * NM], T64[NM * NM];
    };
    uint32_t bitsm[8 * NM * NM];
  };
  double lam_t[NM], lam[NM];
  float ered[kWarps][NM + 2];
  double Ered[NM + 2];
  float featv[kMlpF];
  float mh1[kMlpH];
  float st_min[kWarps], st_max[kWarps], st_tg[kWarps], st_xg[kWarps], st_rowmax[kWarps];
  int wq[NM];
  uint32_t qor[kWarps][NM];
  int kmax, ncorr, nesc, ovf, nonfinite, abort_flag;
  int nesc_slot;                  // escapes listed in the staging slot by the encode pass
  uint32_t* esc_list;             // where (null: not listed), and how many fit
  int esc_cap;
  int64_t bi, bnext;
  int r_pred;
  unsigned nexact;
  int warp_cnt[kWarps];
  int sh32[32];
  int64_t colbase[NM + 1];
  unsigned long long ph[kPhases];   // cycle counters of this CTA (thread 0)
  JacPairs jp;
  unsigned long long mma_bar;     // tcgen05.commit target
  uint32_t mma_phase;             // commits waited for so far (thread 0)
  int mma_pending;                // a wait for products timed out
  uint32_t tmem_base;             // TMEM columns of this CTA (tensor-core Gram)
  BlockMeta m;
  RecLayout lay;
  // the current variable's constants (thread 0 recomputes them when a block
  // of another variable starts) and the eigenvalue sum
  int cvar;
  RowConst crc;
  CorrConst ccc;
  double lam_tr;
  alignas(1024) float ring[kStages][kStageFloats];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after kWaitCycles (the clock is read every 1024 polls).
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    for (int i = 0; i < 1024; ++i)
      if (mbar_try_wait(b, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, unsigned long long* bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_arrive(unsigned long long* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// ---------------------------------------------------------------- tcgen05
// Shared-memory matrix descriptor, no swizzle: start, leading byte offset (the
// K-direction stride between 8x16-byte core matrices), stride byte offset
// (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
               "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void tc_mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
               "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
               : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// 8 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
constexpr uint32_t kTmemCols = 128;

// ---------------------------------------------------------------- chunk geometry
// A block is cut into chunks of zc z-planes x yc y-lines (all x, all t); the
// chunk's tile in shared memory is [t][z][y][x] with bxb x-values per line,
// so row r of the chunk (x fastest) has its t-th value at t * rc + r.
struct Chunks {
  int ncy, ncz, n;
};
__device__ __forceinline__ Chunks chunks_of(const TileArgs& a, const Geom& g) {
  Chunks c;
  c.ncy = (int)cdiv(g.sy, a.yc);
  c.ncz = (int)cdiv(g.sz, a.zc);
  c.n = c.ncy * c.ncz;
  return c;
}
// floor(r / d) for r, d < 2^12 by a multiply-high with m = ceil(2^32 / d)
// (exact while r d < 2^32; m = 0 encodes d = 1).
__device__ __forceinline__ int fdiv(int r, uint32_t m) { return m ? (int)__umulhi((uint32_t)r, m) : r; }

// Row r of chunk c: its dense block row index l (x fastest over the block), or -1.
__device__ __forceinline__ int row_index(const TileArgs& a, const Geom& g, const Chunks& ch, int c, int r, int* xo) {
  const int t2 = fdiv(r, a.mbx);
  const int x = r - t2 * a.bxb;
  const int zl = fdiv(t2, a.myc);
  const int yl = t2 - zl * a.yc;
  const int cz = c / ch.ncy;
  const int y = (c - cz * ch.ncy) * a.yc + yl, z = cz * a.zc + zl;
  *xo = x;
  if (x >= g.sx || y >= g.sy || z >= g.sz) return -1;
  return (z * g.sy + y) * g.sx + x;
}

// Global index of block entry (row l, column j) of a side-0 block.
__device__ __forceinline__ int64_t gidx_plan(const Plan& P, const Geom& g, int64_t l, int j) {
  const int64_t x = l % g.sx, r = l / g.sx;
  const int64_t y = r % g.sy, z = r / g.sy;
  return (int64_t)g.v * P.K + (g.t0 + j) * P.P + ((g.z0 + z) * P.dims[1] + (g.y0 + y)) * P.dims[0] + (g.x0 + x);
}
__device__ __forceinline__ int64_t gidx_row(const TileArgs& a, const Geom& g, int64_t l, int j) {
  const int64_t x = l % g.sx, r = l / g.sx;
  const int64_t y = r % g.sy, z = r / g.sy;
  return (int64_t)g.v * a.P.K + (g.t0 + j) * a.P.P + ((g.z0 + z) * a.P.dims[1] + (g.y0 + y)) * a.P.dims[0] +
         (g.x0 + x);
}

// The two tensor maps of a launch: row tiles [t][z][y][x] for the row-wise
// passes, and the core-matrix tiles of the tensor-core Gram (see pass_gram_tc).
struct Maps {
  const CUtensorMap* row;
  const CUtensorMap* gram;
};
constexpr int kLayoutRow = 0, kLayoutGram = 1;

// True when the block is full and its chunk rows are its rows in order (row l of
// chunk c is l = c rc + r: whole x lines, y chunks that tile the block's y
// extent, whole planes when a chunk holds several), with rc and M multiples of
// 32: then every warp step of the row-wise passes covers 32 consecutive rows
// from a multiple of 32.
__device__ __forceinline__ bool bitmap_rows(const TileArgs& a, const Geom& g) {
  const bool ylines = a.zc == 1 ? g.sy % a.yc == 0 : g.sy == a.yc;
  return g.sx == a.bxb && ylines && g.sz % a.zc == 0 && (a.rc & 31) == 0 && (g.M & 31) == 0;
}

__device__ void issue_chunk(const TileArgs& a, const Maps& tm, TileSmem& S, int64_t bi, const Geom& g,
                            const Chunks& ch, int c, uint32_t& iss, int layout) {
  if (c == 0 && bi == a.withhold) {
    // test hook: the stage is counted as issued but nothing arrives on its
    // barrier, so the wait for it runs out and the call reports a timeout
    ++iss;
    return;
  }
  const int stage = (int)(iss % kStages);
  const int yb = (c % ch.ncy) * a.yc, zb = (c / ch.ncy) * a.zc;
  if (layout == kLayoutGram) {
    // two boxes {4 x, 8 t, 4 x-groups, 16 y, 1 z}: t 0-7 and t 8-15
    if (threadIdx.x == 0) {
      mbar_expect_tx(&S.full[stage], (unsigned)(a.rc * a.bt * 4));
      const int tv = g.v * (int)a.P.dims[3] + (int)g.t0;
      for (int h = 0; h < 2; ++h)
        tma_load_5d(&S.ring[stage][h * 2048], tm.gram, &S.full[stage], 0, tv + 8 * h, (int)(g.x0 / 4),
                    (int)(g.y0 + yb), (int)(g.z0 + zb));
    }
  } else if (a.use_tma) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&S.full[stage], (unsigned)(a.rc * a.bt * 4));
      tma_load_5d(&S.ring[stage][0], tm.row, &S.full[stage], (int)g.x0, (int)(g.y0 + yb), (int)(g.z0 + zb), (int)g.t0,
                  g.v);
    }
  } else {
    // element e of the tile is (t, r) = (e / rc, e % rc), r = (t2, x) with
    // t2 = (zl, yl); divisions by multiply-high (the divisors are below 2^13)
    const Plan& P = a.P;
    const int tot = a.rc * a.bt;
    const int64_t vbase = (int64_t)g.v * P.K;
    const int step = a.cp_pairs ? 2 : 1;
    for (int e = threadIdx.x * step; e < tot; e += kTT * step) {
      const int t = fdiv(e, a.mrc), r = e - t * a.rc;
      const int t2 = fdiv(r, a.mbx), x = r - t2 * a.bxb;
      const int zl = fdiv(t2, a.myc), yl = t2 - zl * a.yc;
      const int64_t gx = g.x0 + x, gy = g.y0 + yb + yl, gz = g.z0 + zb + zl, gt = g.t0 + t;
      const bool ok = gx < P.dims[0] && gy < P.dims[1] && gz < P.dims[2] && gt < P.dims[3];
      const float* src = ok ? a.in + vbase + gt * P.P + (gz * P.dims[1] + gy) * P.dims[0] + gx : a.in;
      // pairs: x even and the field's x extent even, so x + 1 is in the field
      // whenever x is, and both addresses are 8-byte aligned
      if (a.cp_pairs) cp_async8(&S.ring[stage][e], src, ok);
      else cp_async4(&S.ring[stage][e], src, ok);
    }
    cp_async_arrive(&S.full[stage]);
  }
  ++iss;
}

// Waits for the oldest chunk in flight; false (and the CTA's abort flag) on
// timeout.  Thread 0 adds the cycles it waited to the tile-wait counter.
__device__ __forceinline__ bool wait_chunk(TileSmem& S, uint32_t con) {
  const int stage = (int)(con % kStages);
  const long long t0 = threadIdx.x == 0 ? clock64() : 0;
  const bool ok = mbar_wait(&S.full[stage], (con / kStages) & 1u);
  if (!ok) S.abort_flag = 1;
  if (threadIdx.x == 0) S.ph[kPhTileWait] += (unsigned long long)(clock64() - t0);
  return ok;
}

// Ring cursor: chunks [0, pf_cnt) of block pf_blk, in layout pf_layout, are in flight.
struct Cursor {
  uint32_t iss, con;
  int64_t pf_blk;
  int pf_cnt, pf_layout;
};

// Drops chunks in flight that belong to another block.
__device__ void drain(TileSmem& S, Cursor& cu);

// Starts the first chunks of block bi (all threads call).  Chunks already in
// flight for the same block and layout are kept; any others are drained first,
// so the ring never holds more chunks than it has stages.
__device__ void prefetch(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi, const Geom& g,
                         int layout) {
  if (cu.pf_cnt > 0) {
    if (cu.pf_blk == bi && cu.pf_layout == layout) return;
    drain(S, cu);
  }
  const Chunks ch = chunks_of(a, g);
  const int k = ch.n < kStages ? ch.n : kStages;
  for (int c = 0; c < k; ++c) issue_chunk(a, tm, S, bi, g, ch, c, cu.iss, layout);
  cu.pf_blk = bi;
  cu.pf_cnt = k;
  cu.pf_layout = layout;
}

// Drops chunks in flight that belong to another block.
__device__ void drain(TileSmem& S, Cursor& cu) {
  for (int i = 0; i < cu.pf_cnt; ++i) {
    wait_chunk(S, cu.con);
    ++cu.con;
  }
  cu.pf_cnt = 0;
  cu.pf_blk = -1;
  __syncthreads();
}

// Streams every chunk of block bi through the ring, calling body(c, tile) for
// each; all threads call.  Returns false if a wait timed out.
template <class F>
__device__ bool stream_block(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi,
                             const Geom& g, int layout, F&& body) {
  const Chunks ch = chunks_of(a, g);
  const bool match = cu.pf_blk == bi && cu.pf_layout == layout;
  if (!match && cu.pf_cnt > 0) drain(S, cu);
  const int have = match ? cu.pf_cnt : 0;
  const int k = ch.n < kStages ? ch.n : kStages;
  for (int c = have; c < k; ++c) issue_chunk(a, tm, S, bi, g, ch, c, cu.iss, layout);
  cu.pf_cnt = 0;
  cu.pf_blk = -1;
  for (int c = 0; c < ch.n; ++c) {
    wait_chunk(S, cu.con);
    __syncthreads();
    if (S.abort_flag) return false;
    body(c, ch, &S.ring[cu.con % kStages][0]);
    __syncthreads();
    ++cu.con;
    if (c + kStages < ch.n) issue_chunk(a, tm, S, bi, g, ch, c + kStages, cu.iss, layout);
  }
  return true;
}

// ---------------------------------------------------------------- reductions
// Fixed-order CTA reduction of cnt per-thread floats into S.Ered (double).
__device__ void cta_reduce(TileSmem& S, const float* v, int cnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = 0; i < NM + 2; ++i) {
    if (i >= cnt) break;
    float x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(FULL, x, o));
    if (lane == 0) S.ered[warp][i] = x;
  }
  __syncthreads();
  if (tid < cnt) {
    float s = 0.0f;
    for (int w = 0; w < kWarps; ++w) s = __fadd_rn(s, S.ered[w][tid]);
    S.Ered[tid] = (double)s;
  }
  __syncthreads();
}

// After the Gram pass: time-gradient energy sum_rows sum_j (x_{j+1} - x_j)^2
// from the Gram, the row-norm bound n max|x|^2 from the range, and the
// non-finite screen on the diagonal with an exact rescan when it trips (a
// finite block whose squares overflow is not an input error).  All threads.
__device__ void derived_stats(const TileArgs& a, TileSmem& S, const Geom& g, int n) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    float tg = 0.0f;
    bool screen = false;
    for (int j = 0; j < n; ++j) {
      if (!isfinite(S.G32[j * NM + j])) screen = true;
      if (j + 1 < n) tg += S.G32[(j + 1) * NM + j + 1] + S.G32[j * NM + j] - 2.0f * S.G32[j * NM + j + 1];
    }
    float mnn = S.st_min[0], mxx = S.st_max[0];
    for (int w = 1; w < kWarps; ++w) { mnn = fminf(mnn, S.st_min[w]); mxx = fmaxf(mxx, S.st_max[w]); }
    const float am = fmaxf(fabsf(mnn), fabsf(mxx));
    S.st_tg[0] = fmaxf(tg, 0.0f);
    S.st_rowmax[0] = (float)n * am * am;
    S.nonfinite = screen ? 2 : 0;
  }
  __syncthreads();
  if (S.nonfinite == 2) {
    int bad = 0;
    for (int64_t e = tid; e < g.N; e += kTT) {
      const int64_t lt = e / g.M, ls = e - lt * g.M;
      if (!isfinite(__ldg(a.in + gidx_row(a, g, ls, (int)lt)))) bad = 1;
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) S.nonfinite = bad;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Gram pass
// Group g (2 warps) accumulates packed pairs [68 g, 68 g + 68) over every row;
// each group gathers the statistics of every other row.  With `project`, rows
// are first projected onto the current basis (Rayleigh-Ritz matrix).
// NF = 16: the Gram order is 16 and known at compile time (no per-column
// predicates); NF = 0: any order n <= 16.
// Shifted projection of a row onto one basis column (defined with the encode pass).
template <int NF>
__device__ __forceinline__ float project(const float* d, const float* v, float a0, float vsum, int n);

// Gram accumulation order.  The upper triangle is covered by the diagonal
// singles (i, i), i even, and the pairs {(i, j), (i + 1, j)}, i even,
// j = i + 1 .. 15, taken i-major.  Group g keeps pairs 2k + g as accumulators
// acc[2k], acc[2k + 1] (rows i, i + 1) and singles 2k + g as acc[64 + k].
constexpr int kGramPairs = 64, kGramSingles = 8;
static_assert(kGramPairs + kGramSingles / 2 * 2 == 72 && kGramPairs + kGramSingles / 2 == kHalf, "layout");
template <int G>
__device__ __forceinline__ void gram_row(const float (&x)[NM], float (&acc)[kHalf]) {
  int pc = 0, sc = 0;
#pragma unroll
  for (int i = 0; i < NM; i += 2) {
    if ((sc & 1) == G) acc[kGramPairs + (sc >> 1)] = __fmaf_rn(x[i], x[i], acc[kGramPairs + (sc >> 1)]);
    ++sc;
#pragma unroll
    for (int j = i + 1; j < NM; ++j, ++pc) {
      if ((pc & 1) == G) {
        const int q = (pc >> 1) * 2;
        const float2 r = __ffma2_rn(make_float2(x[i], x[i + 1]), make_float2(x[j], x[j]),
                                    make_float2(acc[q], acc[q + 1]));
        acc[q] = r.x;
        acc[q + 1] = r.y;
      }
    }
  }
}
// Entry (i, j) of accumulator q of group grp.
__device__ __forceinline__ void gram_entry(int grp, int q, int& i, int& j) {
  if (q >= kGramPairs) {
    i = j = 2 * (2 * (q - kGramPairs) + grp);
    return;
  }
  int pc = 2 * (q >> 1) + grp;                  // global pair index
  int ib = 0;
  while (pc >= NM - 1 - ib) { pc -= NM - 1 - ib; ib += 2; }
  j = ib + 1 + pc;
  i = ib + (q & 1);
}

template <bool PROJECT, int NF>
__device__ __noinline__ bool pass_gram(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi,
                          const Geom& g) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = tid / kGT, gt = tid % kGT;
  const int n = NF ? NF : g.n;
  float acc[kHalf];
#pragma unroll
  for (int p = 0; p < kHalf; ++p) acc[p] = 0.0f;
  float mn = INFINITY, mx = -INFINITY, xg = 0.0f;
  // full blocks whose chunk rows are the block rows: every row is valid and
  // its x is r mod the block width
  const bool lin = bitmap_rows(a, g);
  const int rc = a.rc, bxb = a.bxb, sx = g.sx;
  const uint32_t mbx = a.mbx;
  const bool ok = stream_block(a, tm, S, cu, bi, g, kLayoutRow, [&](int c, const Chunks& ch, const float* tile) {
    int ii = 0;
    for (int r = gt; r < rc; r += kGT, ++ii) {
      int xx;
      if (lin) {
        xx = r - fdiv(r, mbx) * bxb;
      } else if (row_index(a, g, ch, c, r, &xx) < 0) {
        continue;
      }
      float x[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) x[j] = j < n ? tile[j * rc + r] : 0.0f;
      if (PROJECT) {
        // the coefficients on the current basis, as the encode pass computes them
        const float a0 = x[0];
        float d[NM], cc[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) d[j] = j < n ? __fsub_rn(x[j], a0) : 0.0f;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
          cc[k] = 0.0f;
          if (k < n) {
            float v[NM];
            const float4* vp = reinterpret_cast<const float4*>(&S.VstT[k * NM]);
#pragma unroll
            for (int j4 = 0; j4 < NM / 4; ++j4) {
              const float4 t = vp[j4];
              v[4 * j4 + 0] = t.x; v[4 * j4 + 1] = t.y; v[4 * j4 + 2] = t.z; v[4 * j4 + 3] = t.w;
            }
            cc[k] = project<NF>(d, v, a0, S.vsum[k], n);
          }
        }
#pragma unroll
        for (int k = 0; k < NM; ++k) x[k] = cc[k];
      } else if ((ii & 1) == grp) {
        // per-element statistics: range and x-gradient energy (the time
        // gradient, the row-norm bound and the non-finite screen come from
        // the Gram afterwards)
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            mn = fminf(mn, x[j]);
            mx = fmaxf(mx, x[j]);
          }
        }
        if (xx + 1 < sx) {
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < n) { const float d = tile[j * rc + r + 1] - x[j]; xg = __fmaf_rn(d, d, xg); }
        }
      }
      // entries of rows i, i + 1 (i even) in column j as one packed FMA
      // (each component rounds as __fmaf_rn: the same sums as one FMA per
      // entry); groups take alternate pairs and alternate diagonal singles
      if (grp == 0) gram_row<0>(x, acc);
      else gram_row<1>(x, acc);
    }
  });
  if (!ok) return false;
#pragma unroll
  for (int p = 0; p < kHalf; ++p) {
    float v = acc[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, o));
    if (lane == 0) S.red[warp][p] = v;
  }
  if (!PROJECT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
      xg += __shfl_xor_sync(FULL, xg, o);
    }
    if (lane == 0) {
      S.st_min[warp] = mn; S.st_max[warp] = mx; S.st_xg[warp] = xg;
      S.st_tg[warp] = 0.0f; S.st_rowmax[warp] = 0.0f;
    }
  }
  __syncthreads();
  for (int p = tid; p < kNP; p += kTT) {
    const int gw = (p / kHalf) * 2, pp = p % kHalf;
    const float v = __fadd_rn(S.red[gw][pp], S.red[gw + 1][pp]);
    int i, j;
    gram_entry(p / kHalf, pp, i, j);
    if (i < n && j < n) {
      S.G32[i * NM + j] = v; S.G32[j * NM + i] = v;
      S.G64[i * NM + j] = (double)v; S.G64[j * NM + i] = (double)v;
    }
  }
  __syncthreads();
  if (!PROJECT) derived_stats(a, S, g, n);
  return true;
}

// ---------------------------------------------------------------- tensor-core Gram
// Gram pass on the tensor cores, for chunk boxes of 16 x 16 x 1 x 16.
// The Gram map stages a chunk as [t / 8][y][x / 4][t % 8][x % 4]: each y-pair
// is a subset s of 32 spatial rows, and the tile is the K-major operand of a
// 128-row matrix A whose row m = (t / 8, s, t % 8) holds time step t over the
// 32 rows of subset s (8-row groups 1024 B apart, 4-row K steps 128 B apart,
// no swizzle).  D = A A^T accumulates in TMEM over the chunks of the block;
// the Gram is the sum of its eight diagonal 16 x 16 blocks (one per subset).
// Modes (the operands of each product are exact in the MMA's input type, so
// the products do not depend on how the tensor cores convert FP32):
//   3xTF32  hi = x with its 13 low mantissa bits cleared (in place), lo = x - hi
//           truncated to TF32 (second buffer); D += hi hi^T + hi lo^T + lo hi^T
//           (about 21 bits of each x kept: relative error 2^-21);
//   TF32    D += hi hi^T (10-bit mantissas, relative error 2^-11);
//   BF16X3  x = b0 + b1 + ..., b0 = bf16(x), b1 = bf16(x - b0) (round to
//           nearest even), written as a K-major bf16 operand [t / 8][s][k / 8]
//           [t % 8][k % 8] (core matrices 128 B, K neighbours 128 B apart,
//           8-row groups 512 B apart); D += b0 b0^T + b0 b1^T + b1 b0^T
//           (kind::f16), the three-product split of Henry, Tang and Heinecke
//           (2019): relative error about 2^-16;
//   BF16    D += b0 b0^T (8-bit mantissas, relative error 2^-9).
enum TcMode : int { kTcNone = 0, kTcTf32x3 = 1, kTcTf32 = 2, kTcBf16x3 = 3, kTcBf16 = 4 };
__device__ __forceinline__ float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

__device__ __noinline__ bool pass_gram_tc(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi,
                                          const Geom& g, float* lo) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n;
  const int mode = a.tc_gram;
  const bool bf = mode == kTcBf16x3 || mode == kTcBf16;
  float mn = INFINITY, mx = -INFINITY, xg = 0.0f;
  // D FP32; N = 128 (bits 17-22: N/8), M = 128 (bits 24-28: M/16); A, B TF32
  // (kind::tf32, format 2) or BF16 (kind::f16, format 1), K-major
  const uint32_t fmt = bf ? 1u : 2u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
  uint32_t accum = 0;
  const bool ok = stream_block(a, tm, S, cu, bi, g, kLayoutGram, [&](int c, const Chunks& ch, const float* tile_c) {
    float* tile = const_cast<float*>(tile_c);
    // statistics of the valid elements (read-only pass: neighbours are read)
    for (int gi = tid; gi < 1024; gi += kTT) {
      const int t = (gi >> 9) * 8 + (gi & 7), xc = (gi >> 3) & 3, y = (gi >> 5) & 15;
      if (t < n && y < g.sy) {
        const float4 v = reinterpret_cast<const float4*>(tile)[gi];
        const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int x = xc * 4 + i;
          if (x < g.sx) {
            mn = fminf(mn, xv[i]);
            mx = fmaxf(mx, xv[i]);
            if (x + 1 < g.sx) {
              const float nb = i < 3 ? xv[i + 1] : tile[(gi + 8) * 4];
              const float d = nb - xv[i];
              xg = __fmaf_rn(d, d, xg);
            }
          }
        }
      }
    }
    __syncthreads();
    if (!bf) {
      // split into hi (in place) and, for 3xTF32, lo
      for (int gi = tid; gi < 1024; gi += kTT) {
        const float4 v = reinterpret_cast<const float4*>(tile)[gi];
        float4 h, l;
        h.x = tf32_trunc(v.x); l.x = tf32_trunc(__fsub_rn(v.x, h.x));
        h.y = tf32_trunc(v.y); l.y = tf32_trunc(__fsub_rn(v.y, h.y));
        h.z = tf32_trunc(v.z); l.z = tf32_trunc(__fsub_rn(v.z, h.z));
        h.w = tf32_trunc(v.w); l.w = tf32_trunc(__fsub_rn(v.w, h.w));
        reinterpret_cast<float4*>(tile)[gi] = h;
        if (mode == kTcTf32x3) reinterpret_cast<float4*>(lo)[gi] = l;
      }
    } else {
      // bf16 operands: output row (h, s, kc, tr) holds x = 8 (kc % 2) .. + 7 of
      // y = 2 s + kc / 2 at t = 8 h + tr; b0 in lo[0, 8 KiB), b1 after it
      for (int o = tid; o < 512; o += kTT) {
        const int tr = o & 7, kc = (o >> 3) & 3, sub = (o >> 5) & 7, h = o >> 8;
        const int y = 2 * sub + (kc >> 1), xq = 2 * (kc & 1);
        const int gi = ((h * 16 + y) * 4 + xq) * 8 + tr;
        const float4 v0 = reinterpret_cast<const float4*>(tile)[gi];
        const float4 v1 = reinterpret_cast<const float4*>(tile)[gi + 8];
        const float xv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint32_t p0[4], p1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat16 a0 = __float2bfloat16_rn(xv[2 * i]), c0 = __float2bfloat16_rn(xv[2 * i + 1]);
          const __nv_bfloat16 a1 = __float2bfloat16_rn(__fsub_rn(xv[2 * i], __bfloat162float(a0)));
          const __nv_bfloat16 c1 = __float2bfloat16_rn(__fsub_rn(xv[2 * i + 1], __bfloat162float(c0)));
          p0[i] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(c0) << 16);
          p1[i] = (uint32_t)__bfloat16_as_ushort(a1) | ((uint32_t)__bfloat16_as_ushort(c1) << 16);
        }
        reinterpret_cast<uint4*>(lo)[o] = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        if (mode == kTcBf16x3) reinterpret_cast<uint4*>(lo)[512 + o] = make_uint4(p1[0], p1[1], p1[2], p1[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      if (!bf) {
        const uint32_t ha = smem_u32(tile), la = smem_u32(lo);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t dh = sdesc(ha + ks * 256, 128, 1024), dl = sdesc(la + ks * 256, 128, 1024);
          tc_mma_tf32(S.tmem_base, dh, dh, idesc, accum);
          accum = 1;
          if (mode == kTcTf32x3) {
            tc_mma_tf32(S.tmem_base, dh, dl, idesc, 1);
            tc_mma_tf32(S.tmem_base, dl, dh, idesc, 1);
          }
        }
      } else {
        const uint32_t b0 = smem_u32(lo), b1 = b0 + 8192;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t d0 = sdesc(b0 + ks * 256, 128, 512), d1 = sdesc(b1 + ks * 256, 128, 512);
          tc_mma_f16(S.tmem_base, d0, d0, idesc, accum);
          accum = 1;
          if (mode == kTcBf16x3) {
            tc_mma_f16(S.tmem_base, d0, d1, idesc, 1);
            tc_mma_f16(S.tmem_base, d1, d0, idesc, 1);
          }
        }
      }
      tc_commit(&S.mma_bar);
      // the stage and the operand buffer are reused next: wait for the products
      if (mbar_wait(&S.mma_bar, S.mma_phase & 1u)) {
        ++S.mma_phase;
      } else {
        S.abort_flag = 1;
        S.mma_pending = 1;
      }
    }
    (void)c; (void)ch;
  });
  if (!ok) return false;
  tc_fence_after();
  // read D: warp w holds rows m = 32 w + lane = (t / 8 = w / 2, s = 4 (w % 2) + lane / 8, t % 8 = lane % 8)
  {
    const int half = warp & 1, sl = lane >> 3, tl = lane & 7, h = warp >> 1;
    float v0[8], v1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { v0[i] = 0.0f; v1[i] = 0.0f; }
    const uint32_t tw = S.tmem_base + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float r0[8], r1[8];
      tc_ld8(tw + (uint32_t)((4 * half + q) * 8), r0);
      tc_ld8(tw + (uint32_t)(64 + (4 * half + q) * 8), r1);
      if (sl == q) {
#pragma unroll
        for (int i = 0; i < 8; ++i) { v0[i] = r0[i]; v1[i] = r1[i]; }
      }
    }
    // sum the warp's four subsets: lanes tl, tl + 8, tl + 16, tl + 24
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v0[i] = __fadd_rn(v0[i], __shfl_xor_sync(FULL, v0[i], 8));
      v1[i] = __fadd_rn(v1[i], __shfl_xor_sync(FULL, v1[i], 8));
      v0[i] = __fadd_rn(v0[i], __shfl_xor_sync(FULL, v0[i], 16));
      v1[i] = __fadd_rn(v1[i], __shfl_xor_sync(FULL, v1[i], 16));
    }
    float* part = &S.red[0][0];                 // [h][t % 8][16]
    if (half == 1 && sl == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) { part[(h * 8 + tl) * 16 + i] = v0[i]; part[(h * 8 + tl) * 16 + 8 + i] = v1[i]; }
    }
    tc_fence_before();
    __syncthreads();
    if (half == 0 && sl == 0) {
      const int t = h * 8 + tl;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        S.G32[t * NM + i] = __fadd_rn(v0[i], part[(h * 8 + tl) * 16 + i]);
        S.G32[t * NM + 8 + i] = __fadd_rn(v1[i], part[(h * 8 + tl) * 16 + 8 + i]);
      }
    }
    __syncthreads();
  }
  // symmetric from the upper triangle; FP64 copy; statistics
  for (int e = tid; e < NM * NM; e += kTT) {
    const int i = e / NM, j = e % NM;
    if (i < n && j < n) {
      const float v = i <= j ? S.G32[i * NM + j] : S.G32[j * NM + i];
      S.G64[e] = (double)v;
    }
  }
  __syncthreads();
  for (int e = tid; e < NM * NM; e += kTT) {
    const int i = e / NM, j = e % NM;
    if (i < n && j < n) S.G32[e] = (float)S.G64[e];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    xg += __shfl_xor_sync(FULL, xg, o);
  }
  if (lane == 0) {
    S.st_min[warp] = mn; S.st_max[warp] = mx; S.st_xg[warp] = xg;
    S.st_tg[warp] = 0.0f; S.st_rowmax[warp] = 0.0f;
  }
  if (tid == 0) S.ph[kCntTcGram] += 1;
  __syncthreads();
  derived_stats(a, S, g, n);
  return true;
}

// ---------------------------------------------------------------- orthonormalisation
// First-order orthonormalisation of the eigenvector matrix X (columns = modes;
// all threads), into X64 for the ordering: X <- X + X R / 2, R = I - X^T X.
// The FP32 Jacobi's rotations are orthogonal to a few ulps each, so its
// eigenvectors are orthonormal to about 1e-5; the step takes that to its
// square.  R is formed without rounding error that matters: each product
// a b is split exactly into fl(a b) + fma(a, b, -fl(a b)) and the sums are
// kept as unevaluated pairs (Knuth's two-sum), so R is exact to about 1e-14
// with FP32 arithmetic alone (GB300's FP64 pipe is 1/64 of its FP32 rate);
// the correction X R / 2, of size |R|, and the final rounding need only FP32.
// With `rotate`, X = Vst W first (the Rayleigh-Ritz rotation of the first
// basis, in FP32: its rounding is orthonormalised away with the rest).
__device__ __noinline__ void orth_basis(TileSmem& S, int n, bool rotate) {
  const int tid = threadIdx.x;
  if (rotate) {
    float* X = &S.red[0][0];                    // scratch (>= NM * NM floats)
    static_assert(sizeof(S.red) >= NM * NM * sizeof(float), "scratch");
    for (int e = tid; e < NM * NM; e += kTT) {
      const int i = e / NM, j = e % NM;
      float v = 0.0f;
      if (i < n && j < n)
        for (int k = 0; k < n; ++k) v = __fmaf_rn(S.VstT[k * NM + i], S.Vj[k * NM + j], v);
      X[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < NM * NM; e += kTT) S.Vj[e] = X[e];
    __syncthreads();
  }
  float* R = S.G32;                             // the Gram is not needed any more
  for (int e = tid; e < NM * NM; e += kTT) {
    const int i = e / NM, j = e % NM;
    if (i < n && j < n && i <= j) {
      float sh = 0.0f, sl = 0.0f;
      for (int k = 0; k < n; ++k) {
        const float x = S.Vj[k * NM + i], y = S.Vj[k * NM + j];
        const float ph = __fmul_rn(x, y);
        const float pl = __fmaf_rn(x, y, -ph);  // x y = ph + pl exactly
        const float t = __fadd_rn(sh, ph);
        const float bv = __fsub_rn(t, sh);
        const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(ph, bv));   // sh + ph = t + er
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(er, pl));
      }
      // delta_ij - (sh + sl); 1 - sh is exact for sh in [1/2, 2]
      const float r = i == j ? __fsub_rn(__fsub_rn(1.0f, sh), sl) : -__fadd_rn(sh, sl);
      R[i * NM + j] = r;
      R[j * NM + i] = r;
    }
  }
  __syncthreads();
  float xn[NM * NM / kTT];
  int cnt = 0;
  for (int e = tid; e < NM * NM; e += kTT, ++cnt) {
    const int i = e / NM, j = e % NM;
    xn[cnt] = 0.0f;
    if (i < n && j < n) {
      float c = 0.0f;
      for (int k = 0; k < n; ++k) c = __fmaf_rn(S.Vj[i * NM + k], R[k * NM + j], c);
      xn[cnt] = __fmaf_rn(0.5f, c, S.Vj[e]);
    }
  }
  __syncthreads();
  cnt = 0;
  for (int e = tid; e < NM * NM; e += kTT, ++cnt) {
    const int i = e / NM, j = e % NM;
    if (i < n && j < n) S.X64[e] = (double)xn[cnt];
  }
  __syncthreads();
}

// Sort (stable, descending, lambda < 0 -> 0), sign-normalise, round to f32 (warp 0).
__device__ void order_basis(TileSmem& S, int n, int lane) {
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
    for (int r = 0; r < n; ++r) {
      const double av = fabs(S.X64[r * NM + k]);
      if (av > amax) { amax = av; imax = r; }
    }
    const bool neg = S.X64[imax * NM + k] < 0.0;
    S.lam[pos] = dk;
    double cs = 0.0;
    for (int r = 0; r < NM; ++r) {
      float vf = 0.0f;
      if (r < n) {
        const double v = S.X64[r * NM + k];
        vf = __double2float_rn(neg ? -v : v);
        cs += (double)vf;
      }
      S.VstT[pos * NM + r] = vf;
    }
    S.vsum[pos] = (float)cs;
  }
  if (lane >= n && lane < NM) {
    for (int r = 0; r < NM; ++r) S.VstT[lane * NM + r] = 0.0f;
    S.vsum[lane] = 0.0f;
  }
  __syncwarp();
}

// ---------------------------------------------------------------- row arithmetic
// Coefficient k of one row (shifted projection: sum_j (x_j - x_0) Vst[j][k]
// + x_0 sum_j Vst[j][k], the differences exact when the row carries a large
// common part), quantized with FP64 semantics and dequantized in float.
// The encode, search and exact passes all call this, so all see the same numbers.
// Shifted projection sum_j d_j v_j + a0 vsum in four interleaved partial
// sums (j mod 4), combined as (s0 + s1) + (s2 + s3): the one order every pass
// uses for the coefficients.
// Order 16 (NF = NM): the partial-sum pairs (s0, s1), (s2, s3) as packed
// FP32 FMAs (each component rounds as __fmaf_rn: the same numbers).
template <int NF>
__device__ __forceinline__ float project(const float* d, const float* v, float a0, float vsum, int n) {
  if (NF == NM) {
    float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j4 = 0; j4 < NM / 4; ++j4) {
      s01 = __ffma2_rn(make_float2(d[4 * j4 + 0], d[4 * j4 + 1]), make_float2(v[4 * j4 + 0], v[4 * j4 + 1]), s01);
      s23 = __ffma2_rn(make_float2(d[4 * j4 + 2], d[4 * j4 + 3]), make_float2(v[4 * j4 + 2], v[4 * j4 + 3]), s23);
    }
    return __fmaf_rn(a0, vsum, __fadd_rn(__fadd_rn(s01.x, s01.y), __fadd_rn(s23.x, s23.y)));
  }
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
  for (int j4 = 0; j4 < NM / 4; ++j4) {
    if (4 * j4 + 0 < n) s0 = __fmaf_rn(d[4 * j4 + 0], v[4 * j4 + 0], s0);
    if (4 * j4 + 1 < n) s1 = __fmaf_rn(d[4 * j4 + 1], v[4 * j4 + 1], s1);
    if (4 * j4 + 2 < n) s2 = __fmaf_rn(d[4 * j4 + 2], v[4 * j4 + 2], s2);
    if (4 * j4 + 3 < n) s3 = __fmaf_rn(d[4 * j4 + 3], v[4 * j4 + 3], s3);
  }
  return __fmaf_rn(a0, vsum, __fadd_rn(__fadd_rn(s0, s1), __fadd_rn(s2, s3)));
}

template <int NF>
__device__ __forceinline__ float coeff_q(const TileSmem& S, const float* d, float a0, int n_, int k,
                                         const RowConst& rc, int32_t& q, int& ovf) {
  const int n = NF ? NF : n_;
  const float4* vp = reinterpret_cast<const float4*>(&S.VstT[k * NM]);
  float v[NM];
#pragma unroll
  for (int j4 = 0; j4 < NM / 4; ++j4) {
    const float4 t = vp[j4];
    v[4 * j4 + 0] = t.x; v[4 * j4 + 1] = t.y; v[4 * j4 + 2] = t.z; v[4 * j4 + 3] = t.w;
  }
  const float c = project<NF>(d, v, a0, S.vsum[k], n);
  q = quant_exact(c, rc.delta, rc.inv_delta, ovf);
  return __fmul_rn(__int2float_rn(q), rc.delta_f);
}

__device__ __forceinline__ void shifted(const float* x, float* d) {
#pragma unroll
  for (int j = 0; j < NM; ++j) d[j] = __fsub_rn(x[j], x[0]);
}

// acc[j] <- fma(ch[k], Vst[j][k], acc[j]) for one k (decode contract order).
__device__ __forceinline__ void row_decode_step(const TileSmem& S, int k, float chk, float* acc) {
  const float4* vp = reinterpret_cast<const float4*>(&S.VstT[k * NM]);
  const float2 c2 = make_float2(chk, chk);
#pragma unroll
  for (int j4 = 0; j4 < NM / 4; ++j4) {
    const float4 v = vp[j4];
    const float2 a = __ffma2_rn(c2, make_float2(v.x, v.y), make_float2(acc[4 * j4 + 0], acc[4 * j4 + 1]));
    const float2 b = __ffma2_rn(c2, make_float2(v.z, v.w), make_float2(acc[4 * j4 + 2], acc[4 * j4 + 3]));
    acc[4 * j4 + 0] = a.x; acc[4 * j4 + 1] = a.y;
    acc[4 * j4 + 2] = b.x; acc[4 * j4 + 3] = b.y;
  }
}


// Bit-matrix transpose across a warp (lane i's bit j becomes lane j's bit i):
// five butterfly stages, each swapping the off-diagonal halves of the blocks.
__device__ __forceinline__ uint32_t warp_transpose_bits(uint32_t v, int lane) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const uint32_t lo = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t t = __shfl_xor_sync(FULL, v, s);
    v = (lane & s) ? ((v & ~lo) | ((t >> s) & lo)) : ((v & lo) | ((t << s) & ~lo));
  }
  return v;
}

// ---------------------------------------------------------------- encode pass
// Projection, quantization and decode at rank r, q into the CTA scratch,
// corrections into k8/k32; with `check`, FP32 estimates of E(r-1), E(r) land
// in S.Ered[0], S.Ered[1].  One row per thread; the column loop is not
// unrolled (r is small), and each basis row is read once per column for both
// the projection and the decode step.  Column widths: OR of zigzag(q) over
// the warp (same bit width as the maximum), kept by lane k for column k, into S.qor.
// SPARSE (pointwise bound, bitmap rows): k8 is written only for the elements
// whose correction may be nonzero, and the record reads k8 through the
// nonzero-correction bitmap; escapes cannot be listed from such a k8, so a
// block that has any is encoded again without SPARSE.
template <int NF, bool SPARSE>
__device__ __noinline__ bool pass_encode(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi,
                            const Geom& g, int r, bool check, const RowConst& rcst, const CorrConst& cc, bool pointwise,
                            int32_t* qs, int8_t* k8, int32_t* k32, uint32_t* bits) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = NF ? NF : g.n;
  // full blocks whose chunk rows are the block rows in order: each warp step
  // covers 32 consecutive rows starting at a multiple of 32, so a ballot per
  // column is one word of the nonzero-correction bitmap (element e -> bit e)
  const bool use_bits = bitmap_rows(a, g);
  // the constants by value: the loop's stores cannot be assumed not to alias them
  const RowConst rq = rcst;
  const CorrConst cq = cc;
  uint32_t qor_lane = 0;   // lane k: OR of zigzag(q) of column k over this warp's rows
  if (tid == 0) { S.kmax = 0; S.ncorr = 0; S.nesc = 0; S.nesc_slot = 0; }
  __syncthreads();
  float e1 = 0.0f, e2 = 0.0f;
  float2 e1v = make_float2(0.0f, 0.0f), e2v = make_float2(0.0f, 0.0f);   // order 16: even / odd elements
  int nc = 0, ne = 0, ovf = 0;
  uint32_t kmx = 0;
  const int M = (int)g.M, Lq = (int)align_up(g.L, 4), rc = a.rc;
  const bool ok = stream_block(a, tm, S, cu, bi, g, kLayoutRow, [&](int c, const Chunks& ch, const float* tile) {
    for (int rb = 0; rb < rc; rb += kTT) {          // same trip count in every lane
      const int rr = rb + tid;
      int xx = 0;
      const int l = rr < rc ? (use_bits ? c * rc + rr : row_index(a, g, ch, c, rr, &xx)) : -1;
      const bool valid = l >= 0;
      const float* xr = tile + (valid ? rr : 0);
      const float a0 = valid ? xr[0] : 0.0f;
      float d[NM], acc[NM];
      // order 16: element pairs as packed FMAs; fma(a, -1, x) rounds as x - a
      const float2 m1 = make_float2(-1.0f, -1.0f);
      auto x2 = [&](int j2) { return make_float2(xr[2 * j2 * rc], xr[(2 * j2 + 1) * rc]); };
      if (NF == NM && valid) {
#pragma unroll
        for (int j2 = 0; j2 < NM / 2; ++j2) {
          const float2 t = __ffma2_rn(make_float2(a0, a0), m1, x2(j2));
          d[2 * j2] = t.x;
          d[2 * j2 + 1] = t.y;
          acc[2 * j2] = 0.0f;
          acc[2 * j2 + 1] = 0.0f;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          d[j] = (valid && j < n) ? __fsub_rn(xr[j * rc], a0) : 0.0f;
          acc[j] = 0.0f;
        }
      }
#pragma unroll 1
      for (int k = 0; k < r; ++k) {
        float v[NM];
        const float4* vp = reinterpret_cast<const float4*>(&S.VstT[k * NM]);
#pragma unroll
        for (int j4 = 0; j4 < NM / 4; ++j4) {
          const float4 t = vp[j4];
          v[4 * j4 + 0] = t.x; v[4 * j4 + 1] = t.y; v[4 * j4 + 2] = t.z; v[4 * j4 + 3] = t.w;
        }
        const float cf = project<NF>(d, v, a0, S.vsum[k], n);
        const int32_t q = quant_exact(cf, rq.delta, rq.inv_delta, ovf);
        if (valid) qs[k * Lq + l] = q;
        const uint32_t wor = __reduce_or_sync(FULL, valid ? zigzag(q) : 0u);
        if (lane == k) qor_lane |= wor;
        const float chk = __fmul_rn(__int2float_rn(q), rq.delta_f);
        if (check && k == r - 1 && valid) {
          if (NF == NM) {
#pragma unroll
            for (int j2 = 0; j2 < NM / 2; ++j2) {
              const float2 dd = __ffma2_rn(make_float2(acc[2 * j2], acc[2 * j2 + 1]), m1, x2(j2));
              e1v = __ffma2_rn(dd, dd, e1v);
            }
          } else {
#pragma unroll
            for (int j = 0; j < NM; ++j)
              if (j < n) { const float dd = __fsub_rn(xr[j * rc], acc[j]); e1 = __fmaf_rn(dd, dd, e1); }
          }
        }
#pragma unroll
        for (int j2 = 0; j2 < NM / 2; ++j2) {
          // decode step, two elements per packed FMA (each as __fmaf_rn)
          const float2 t = __ffma2_rn(make_float2(chk, chk), make_float2(v[2 * j2], v[2 * j2 + 1]),
                                      make_float2(acc[2 * j2], acc[2 * j2 + 1]));
          acc[2 * j2] = t.x;
          acc[2 * j2 + 1] = t.y;
        }
      }
      if (SPARSE && valid) {
        // elements with |fl(x - xhat)| < eb (rounded down) need no correction
        // (the first test of the decision); the others are decided one by one
        uint32_t cand = 0;
        if (NF == NM) {
#pragma unroll
          for (int j2 = 0; j2 < NM / 2; ++j2) {
            const float2 R = __ffma2_rn(make_float2(acc[2 * j2], acc[2 * j2 + 1]), m1, x2(j2));
            if (check) e2v = __ffma2_rn(R, R, e2v);
            cand |= (corr_candidate(R.x, cq) ? 1u : 0u) << (2 * j2);
            cand |= (corr_candidate(R.y, cq) ? 1u : 0u) << (2 * j2 + 1);
          }
        } else {
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            if (j < n) {
              const float R = __fsub_rn(xr[j * rc], acc[j]);
              if (check) e2 = __fmaf_rn(R, R, e2);
              cand |= (corr_candidate(R, cq) ? 1u : 0u) << j;
            }
          }
        }
        uint32_t nzb = 0, escm = 0;
        while (cand) {
          const int jj = __ffs(cand) - 1;
          cand &= cand - 1;
          float aj = acc[0];
#pragma unroll
          for (int j = 1; j < NM; ++j) aj = (j == jj) ? acc[j] : aj;
          const int32_t k = corr_decide(xr[jj * rc], aj, cq);
          const int e = jj * M + l;
          const bool big = k < -127 || k > 127;            // includes escapes
          k8[e] = big ? (int8_t)-128 : (int8_t)k;
          if (big) k32[e] = k;
          escm |= (k == kEscape ? 1u : 0u) << jj;
          nc += k != 0 ? 1 : 0;
          kmx |= k == kEscape ? 0u : zigzag(k);
          nzb |= (k != 0 && k != kEscape ? 1u : 0u) << jj;
        }
        if (escm) {
          // rare: the row's escapes, listed for the deferred packer (in no
          // particular order)
          ne += __popc(escm);
          uint32_t* const el = S.esc_list;
          if (el) {
            for (uint32_t em = escm; em; em &= em - 1) {
              const int i = atomicAdd(&S.nesc_slot, 1);
              if (i < S.esc_cap) el[i] = (uint32_t)((__ffs(em) - 1) * M + l);
            }
          }
        }
        // lane j gets column j's word of the bitmap (this warp's 32 rows)
        const uint32_t mk = warp_transpose_bits(nzb, lane);
        if (lane < n) bits[(lane * M + (l - lane)) >> 5] = mk;
      } else if (valid) {
        // corrections: every element decided first without branches (so they
        // interleave); the few the FP32 evaluation leaves open take the FP64 path
        int32_t kv[NM];
        uint32_t unsure = 0;
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          kv[j] = 0;
          if (j < n) {
            const float xj = xr[j * rc];
            if (check) { const float dd = __fsub_rn(xj, acc[j]); e2 = __fmaf_rn(dd, dd, e2); }
            if (pointwise) {
              bool u;
              kv[j] = corr_fast(xj, acc[j], cq, &u);
              unsure |= (u ? 1u : 0u) << j;
            }
          }
        }
        while (unsure) {
          const int jj = __ffs(unsure) - 1;
          unsure &= unsure - 1;
          float aj = acc[0];
#pragma unroll
          for (int j = 1; j < NM; ++j) aj = (j == jj) ? acc[j] : aj;
          const int32_t v = corr_slow(xr[jj * rc], aj, cq);
#pragma unroll
          for (int j = 0; j < NM; ++j) kv[j] = (j == jj) ? v : kv[j];
        }
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            const int e = j * M + l;
            const int32_t k = kv[j];
            const bool big = k < -127 || k > 127;            // includes escapes
            k8[e] = big ? (int8_t)-128 : (int8_t)k;
            if (big) k32[e] = k;
            ne += k == kEscape ? 1 : 0;
            nc += k != 0 ? 1 : 0;                             // escapes taken out below
            kmx |= k == kEscape ? 0u : zigzag(k);             // OR: same bit width as the maximum
          }
        }
        if (use_bits) {
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            if (j < n) {
              const unsigned mk = __ballot_sync(FULL, kv[j] != 0 && kv[j] != kEscape);
              if (lane == 0) bits[(j * M + l) >> 5] = mk;
            }
          }
        }
      }
    }
  });
  if (!ok) return false;
  nc -= ne;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nc += __shfl_xor_sync(FULL, nc, o);
    ne += __shfl_xor_sync(FULL, ne, o);
    kmx |= __shfl_xor_sync(FULL, kmx, o);
    ovf |= __shfl_xor_sync(FULL, ovf, o);
  }
  if (lane == 0) {
    if (nc) atomicAdd(&S.ncorr, nc);
    if (ne) atomicAdd(&S.nesc, ne);
    if (kmx) atomicOr(reinterpret_cast<unsigned int*>(&S.kmax), kmx);
    if (ovf) S.ovf = 1;
  }
  if (lane < NM) S.qor[warp][lane] = qor_lane;
  __syncthreads();
  if (tid < NM) {
    uint32_t o = 0;
    for (int w = 0; w < kWarps; ++w) o |= S.qor[w][tid];
    S.wq[tid] = tid < r ? bit_width(o) : 0;
  }
  e1 = __fadd_rn(e1, __fadd_rn(e1v.x, e1v.y));
  e2 = __fadd_rn(e2, __fadd_rn(e2v.x, e2v.y));
  const float ev[2] = {e1, e2};
  if (check) cta_reduce(S, ev, 2);
  else __syncthreads();
  return true;
}

// E(r) for every r in [0, rcap] (FP32 estimates into S.Ered).
template <int NF>
__device__ __noinline__ bool pass_all_errors(const TileArgs& a, const Maps& tm, TileSmem& S, Cursor& cu, int64_t bi,
                                const Geom& g, int rcap, const RowConst& rcst, int& ovf) {
  const int tid = threadIdx.x, n = NF ? NF : g.n;
  float E[NM + 1];
#pragma unroll
  for (int r = 0; r <= NM; ++r) E[r] = 0.0f;
  const bool ok = stream_block(a, tm, S, cu, bi, g, kLayoutRow, [&](int c, const Chunks& ch, const float* tile) {
    for (int rr = tid; rr < a.rc; rr += kTT) {
      int xx;
      const int l = row_index(a, g, ch, c, rr, &xx);
      if (l < 0) continue;
      const float* xr = tile + rr;
      const float a0 = xr[0];
      float d[NM];
      float acc[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        acc[j] = 0.0f;
        d[j] = 0.0f;
        if (j < n) {
          const float xj = xr[j * a.rc];
          d[j] = __fsub_rn(xj, a0);
          E[0] = __fmaf_rn(xj, xj, E[0]);
        }
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        if (k < rcap) {
          int32_t q;
          const float chk = coeff_q<NF>(S, d, a0, n, k, rcst, q, ovf);
          row_decode_step(S, k, chk, acc);
#pragma unroll
          for (int j = 0; j < NM; ++j)
            if (j < n) { const float dd = __fsub_rn(xr[j * a.rc], acc[j]); E[k + 1] = __fmaf_rn(dd, dd, E[k + 1]); }
        }
      }
    }
  });
  if (!ok) return false;
  cta_reduce(S, E, rcap + 1);
  return true;
}

// FP64 evaluation of E(r) in the fixed order of the definition (per column,
// rows in chunks of 32, chunk sums in order, column sums in order), from the
// input in global memory.  Used only when the FP32 estimate cannot decide.
// Thread t takes chunk t of each group of kTT chunks: it decodes each of its
// rows once and accumulates every column's chunk sum; the chunk sums of a
// group wait in the staging ring (idle between passes) and thread j adds
// column j's in chunk order.
__device__ __noinline__ double exact_error(const TileArgs& a, TileSmem& S, const Geom& g, int r, const RowConst& rcst) {
  const int tid = threadIdx.x, n = g.n;
  const int64_t nch = cdiv(g.L, 32);
  double* part = reinterpret_cast<double*>(&S.ring[0][0]);      // kTT chunks x NM columns
  static_assert(sizeof(S.ring) >= kTT * NM * sizeof(double), "scratch");
  double colsum = 0.0;
  for (int64_t c0 = 0; c0 < nch; c0 += kTT) {
    const int64_t c = c0 + tid;
    if (c < nch) {
      double pc[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) pc[j] = 0.0;
      const int64_t l1 = (c + 1) * 32 < g.L ? (c + 1) * 32 : g.L;
      for (int64_t l = c * 32; l < l1; ++l) {
        float x[NM];
#pragma unroll
        for (int jj = 0; jj < NM; ++jj) x[jj] = jj < n ? __ldg(a.in + gidx_row(a, g, l, jj)) : 0.0f;
        float d[NM];
        shifted(x, d);
        int ovf = 0;
        float acc[NM];
#pragma unroll
        for (int jj = 0; jj < NM; ++jj) acc[jj] = 0.0f;
        for (int k = 0; k < r; ++k) {
          int32_t q;
          const float chk = coeff_q<0>(S, d, x[0], n, k, rcst, q, ovf);
          row_decode_step(S, k, chk, acc);
        }
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          if (j < n) {
            const double dd = __dsub_rn((double)x[j], (double)acc[j]);
            pc[j] = __fma_rn(dd, dd, pc[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NM; ++j) part[tid * NM + j] = pc[j];
    }
    __syncthreads();
    if (tid < n) {
      const int64_t cend = (nch - c0) < kTT ? (nch - c0) : kTT;
      for (int64_t cc = 0; cc < cend; ++cc) colsum = __dadd_rn(colsum, part[cc * NM + tid]);
    }
    __syncthreads();
  }
  if (tid < n) S.lam_t[tid] = colsum;           // lam_t is free once the basis is ordered
  // the ring's next writer is the copy engine (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  double E = 0.0;
  for (int j = 0; j < n; ++j) E = __dadd_rn(E, S.lam_t[j]);
  __syncthreads();
  return E;
}

__device__ bool decide_pass(const TileArgs& a, TileSmem& S, const Geom& g, int r, double E32, double bnd, double el2,
                            const RowConst& rcst) {
  const double lo = E32 / (1.0 + bnd), hi = E32 / (1.0 - bnd);
  if (hi < el2 * (1.0 - 1e-12)) return true;
  if (lo > el2 * (1.0 + 1e-12)) return false;
  if (threadIdx.x == 0) S.nexact += 1;
  return exact_error(a, S, g, r, rcst) <= el2;
}

// ---------------------------------------------------------------- rank prediction
// Warp 0: eigenvalue-tail rank estimate E(r) ~ sum_{i>=r} lambda_i + r L delta^2/12
// and the 32 block features, one per lane (FP32; they only steer a prediction
// that is then checked exactly).
__device__ __noinline__ int predict_rank(const TileArgs& a, TileSmem& S, const Geom& g, int64_t bi, int rcap, double el2,
                            double delta, int lane) {
  const int n = g.n;
  double t = lane < n ? S.lam[lane] : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_down_sync(FULL, t, o);
    if (lane + o < 32) t += y;
  }
  const double qn = (double)g.L * delta * delta / 12.0;
  const bool ok = lane <= rcap && (lane < n ? t : 0.0) + lane * qn <= el2;
  const unsigned m = __ballot_sync(FULL, ok);
  const int rp = m ? (__ffs(m) - 1) : rcap;
  const double tot = __shfl_sync(FULL, t, 0);
  const double l0 = S.lam[0];
  float mn = S.st_min[0], mx = S.st_max[0], tg = 0.0f, xg = 0.0f;
  for (int w = 0; w < kWarps; ++w) {
    mn = fminf(mn, S.st_min[w]); mx = fmaxf(mx, S.st_max[w]);
    tg += S.st_tg[w]; xg += S.st_xg[w];
  }
  const float tot_f = (float)(tot > 0.0 ? tot : 1e-30);
  const float el2_f = (float)el2;
  float f = 0.0f;
  if (lane == 0) f = log10f(tot_f / el2_f + 1e-30f);
  const double tr = __shfl_sync(FULL, t, (lane - 1) & 31);
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
  __syncwarp();
  return rp;
}

// ---------------------------------------------------------------- record
// Each warp compacts a contiguous range of [0, N) in steps of 512 elements,
// 16 consecutive per lane from one 16-byte load of k8: elements for which
// sel(k8[e], e) holds get consecutive indices in element order, and
// emit(e, index) writes them.  k8 is 16-byte aligned; reads stay below
// align16(N).
template <class Sel, class Emit>
__device__ void compact16(TileSmem& S, const int8_t* k8, int N, Sel sel, Emit emit) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int per = (int)(cdiv(cdiv(N, kWarps), 512) * 512);
  const int b0 = warp * per;
  const int b1 = (b0 + per) < N ? (b0 + per) : N;
  auto mask16 = [&](int e0) -> uint32_t {
    uint32_t m = 0;
    if (e0 < b1) {
      const uint4 w = *reinterpret_cast<const uint4*>(k8 + e0);
      const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int8_t b = (int8_t)(wd[i >> 2] >> (8 * (i & 3)));
        if (e0 + i < b1 && sel(b, e0 + i)) m |= 1u << i;
      }
    }
    return m;
  };
  int cnt = 0;
  int s0 = b0;
  for (; s0 + 3 * 512 < b1; s0 += 4 * 512) {       // four loads in flight
    const uint32_t m0 = mask16(s0 + lane * 16), m1 = mask16(s0 + 512 + lane * 16);
    const uint32_t m2 = mask16(s0 + 1024 + lane * 16), m3 = mask16(s0 + 1536 + lane * 16);
    cnt += __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
  }
  for (; s0 < b1; s0 += 512) cnt += __popc(mask16(s0 + lane * 16));
  cnt = __reduce_add_sync(FULL, cnt);
  if (lane == 0) S.warp_cnt[warp] = cnt;
  __syncthreads();
  int base = 0;
  for (int w = 0; w < warp; ++w) base += S.warp_cnt[w];
  for (int s0 = b0; s0 < b1; s0 += 512) {        // second read: mostly L1 hits
    uint32_t m = mask16(s0 + lane * 16);
    const int c = __popc(m);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    int idx = base + incl - c;
    while (m) {
      const int i = __ffs(m) - 1;
      m &= m - 1;
      emit(s0 + lane * 16 + i, idx++);
    }
    base += __shfl_sync(FULL, incl, 31);
  }
  __syncthreads();
}

// Packs 32 consecutive w-bit values per task into exactly w words.
__device__ __forceinline__ void flush32(uint64_t& acc, int& nbits, uint32_t* dst, int& wo) {
  if (nbits >= 32) { dst[wo++] = (uint32_t)acc; acc >>= 32; nbits -= 32; }
}

// ---------------------------------------------------------------- record packing
// The packing steps after the stored basis, shared by the record writer of the
// tile kernel and the deferred packer (k_pack_tile).  All threads of a
// kTT-thread CTA call them.

// 32 values below 2^W into exactly W words, W known at compile time: every
// shift and word boundary is fixed, two instructions a value.
template <int W>
__device__ __forceinline__ void pack32_fixed(uint32_t* dst, const uint32_t (&z)[32]) {
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int bit = i * W, off = bit & 31;
    acc |= z[i] << off;
    if (off + W >= 32) {
      dst[bit >> 5] = acc;
      acc = off + W > 32 ? z[i] >> (32 - off) : 0u;
    }
  }
}
// pack32_fixed<w> for w in [W, kMaxFixedW]; false for other widths.
constexpr int kMaxFixedW = 25;
template <int W = 1>
__device__ __forceinline__ bool pack32_width(uint32_t* dst, const uint32_t (&z)[32], int w) {
  if constexpr (W > kMaxFixedW) {
    return false;
  } else {
    if (w == W) {
      pack32_fixed<W>(dst, z);
      return true;
    }
    return pack32_width<W + 1>(dst, z, w);
  }
}

// q columns: 32 consecutive values of one column per task -> exactly w words.
// qs holds column c at qs + c * align_up(L, 4).  FIXED: full tasks go through
// the compile-time-width packers (the deferred packer; the per-block kernel
// keeps the smaller generic loop).
template <bool FIXED = false>
__device__ __forceinline__ void pack_q(uint32_t* qw, const int32_t* qs, const uint8_t* wq, const int64_t* colbase,
                                       int rr, int64_t L) {
  const int runs = (int)cdiv(L, 32);
  const int64_t Lq = align_up(L, 4);
  for (int task = threadIdx.x; task < runs * rr; task += kTT) {
    const int c = task / runs;
    const int first = (task - c * runs) * 32;
    const int wdt = wq[c];
    if (wdt == 0) continue;
    const int32_t* col = qs + (int64_t)c * Lq + first;
    const int cnt = (int)((L - first) < 32 ? (L - first) : 32);
    uint32_t* dst = qw + colbase[c] + (first / 32) * wdt;
    uint32_t z[32];
    if (cnt == 32) {
      const uint4* cv = reinterpret_cast<const uint4*>(col);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 v = cv[i];
        z[4 * i + 0] = zigzag((int32_t)v.x);
        z[4 * i + 1] = zigzag((int32_t)v.y);
        z[4 * i + 2] = zigzag((int32_t)v.z);
        z[4 * i + 3] = zigzag((int32_t)v.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) z[i] = i < cnt ? zigzag(col[i]) : 0u;
    }
    if (FIXED && cnt == 32 && pack32_width(dst, z, wdt)) continue;
    uint64_t acc = 0;
    int nbits = 0, wo = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (i < cnt) {
        acc |= (uint64_t)z[i] << nbits;
        nbits += wdt;
        flush32(acc, nbits, dst, wo);
      }
    }
    if (nbits > 0) dst[wo] = (uint32_t)acc;
  }
}

// Dense corrections: 32 elements of wk bits per task -> exactly wk words.
// With the bitmap (bits != nullptr) k8 counts only where a bit is set.
template <bool FIXED = false>
__device__ __forceinline__ void pack_dense(uint32_t* cw, const int8_t* k8, const int32_t* k32, const uint32_t* bits,
                                           int wk, int64_t N) {
  const int64_t runs = cdiv(N, 32);
  for (int64_t task = threadIdx.x; task < runs; task += kTT) {
    const int64_t first = task * 32;
    const int cnt = (int)((N - first) < 32 ? (N - first) : 32);
    uint32_t* dst = cw + task * wk;
    const uint32_t bw = bits ? bits[task] : 0xFFFFFFFFu;
    if (FIXED && cnt == 32 && wk <= kMaxFixedW) {
      // no k32 values here (corrections below 64)
      const uint4* kv4 = reinterpret_cast<const uint4*>(k8 + first);
      const uint4 w0 = kv4[0], w1 = kv4[1];
      const uint32_t wd[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      uint32_t z[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        z[i] = (bw >> i) & 1u ? zigzag((int32_t)(int8_t)(wd[i >> 2] >> (8 * (i & 3)))) : 0u;
      pack32_width(dst, z, wk);
      continue;
    }
    int8_t kb[32];
    if (cnt == 32) {
      const uint4* kv4 = reinterpret_cast<const uint4*>(k8 + first);
      const uint4 w0 = kv4[0], w1 = kv4[1];
      const uint32_t wd[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int i = 0; i < 32; ++i) kb[i] = (int8_t)(wd[i >> 2] >> (8 * (i & 3)));
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) kb[i] = i < cnt ? k8[first + i] : (int8_t)0;
    }
    uint64_t acc = 0;
    int nbits = 0, wo = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (i < cnt) {
        int32_t kv = (bw >> i) & 1u ? kb[i] : 0;
        if (kv == -128) kv = k32[first + i];
        acc |= (uint64_t)(kv == kEscape ? 0u : zigzag(kv)) << nbits;
        nbits += wk;
        flush32(acc, nbits, dst, wo);
      }
    }
    if (nbits > 0) dst[wo] = (uint32_t)acc;
  }
}

// Entry list (element indices, in element order) from the nonzero-correction
// bitmap: warp w takes a contiguous range of words, 32 at a step (one per lane,
// so the lanes' counts are alike); a warp scan places each word's entries.
// warp_cnt: kWarps ints of shared scratch.
__device__ __forceinline__ void bitmap_list(uint32_t* list, const uint32_t* bits, int64_t N, int64_t ncorr,
                                            int* warp_cnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (int)(N / 32);
  const int per_w = (int)cdiv(nw, kWarps * 32) * 32;
  const int wb = warp * per_w, we = (wb + per_w) < nw ? (wb + per_w) : nw;
  int cnt = 0;
  for (int w = wb + lane; w < we; w += 32) cnt += __popc(bits[w]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
  if (lane == 0) warp_cnt[warp] = cnt;
  __syncthreads();
  int base = 0;
  for (int i = 0; i < warp; ++i) base += warp_cnt[i];
  for (int w0 = wb; w0 < we; w0 += 32) {
    const int w = w0 + lane;
    uint32_t mk = w < we ? bits[w] : 0u;
    const int c = __popc(mk);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    int idx = base + incl - c;
    base += __shfl_sync(FULL, incl, 31);
    while (mk) {
      const int b = __ffs(mk) - 1;
      mk &= mk - 1;
      if (idx < ncorr) list[idx] = (uint32_t)(w * 32 + b);   // the count and the bits agree
      ++idx;
    }
  }
  __syncthreads();
}

// Sparse corrections: 32 entries of ib + wk bits per task -> exactly ib + wk words.
template <bool FIXED = false>
__device__ __forceinline__ void pack_sparse(uint32_t* cw, const uint32_t* list, const int8_t* k8, const int32_t* k32,
                                            int ib, int wk, int64_t nc) {
  const int W = ib + wk;
  for (int64_t task = threadIdx.x; task < cdiv(nc, 32); task += kTT) {
    const int64_t first = task * 32;
    const int cnt = (int)((nc - first) < 32 ? (nc - first) : 32);
    uint32_t* dst = cw + task * W;
    // all 32 entries, then all 32 correction bytes, before the bit packing
    uint32_t ee[32];
    if (cnt == 32) {
      const uint4* lv = reinterpret_cast<const uint4*>(list + first);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint4 v = lv[i];
        ee[4 * i + 0] = v.x; ee[4 * i + 1] = v.y; ee[4 * i + 2] = v.z; ee[4 * i + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) ee[i] = i < cnt ? list[first + i] : 0u;
    }
    int8_t kb[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) kb[i] = i < cnt ? k8[ee[i]] : (int8_t)0;
    if (FIXED && cnt == 32 && W <= kMaxFixedW) {
      // no k32 values here (corrections below 64); an entry is its index,
      // then its correction, in W <= kMaxFixedW bits
#pragma unroll
      for (int i = 0; i < 32; ++i) ee[i] |= zigzag((int32_t)kb[i]) << ib;
      pack32_width(dst, ee, W);
      continue;
    }
    uint64_t acc = 0;
    int nbits = 0, wo = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      if (i < cnt) {
        const int32_t kv = kb[i] == (int8_t)-128 ? k32[ee[i]] : (int32_t)kb[i];
        acc |= (uint64_t)ee[i] << nbits;
        nbits += ib;
        flush32(acc, nbits, dst, wo);
        acc |= (uint64_t)zigzag(kv) << nbits;
        nbits += wk;
        flush32(acc, nbits, dst, wo);
      }
    }
    if (nbits > 0) dst[wo] = (uint32_t)acc;
  }
}

// Zeroes the 16-byte words of rec that hold padding between sections (below
// `limit`), to be written over by the sections themselves after a barrier.
__device__ __forceinline__ void zero_padding(uint8_t* rec, const RecLayout& lay, const BlockMeta& m, int n,
                                             int64_t qwords, int64_t limit) {
  const int rr = m.r;
  const int64_t ends[6] = {lay.off_wq + rr, lay.off_v + (int64_t)n * rr * 4, lay.off_q + qwords * 4,
                           lay.off_c + lay.corr_words * 4, lay.off_ei + (int64_t)m.nesc * 4,
                           lay.off_ev + (int64_t)m.nesc * 4};
  for (int i = 0; i < 6; ++i) {
    const int64_t w = ends[i] / 16 * 16;
    if (w < m.nbytes && w < limit) *reinterpret_cast<uint4*>(rec + w) = make_uint4(0, 0, 0, 0);
  }
}

// Deferred packing: a record whose q columns, nonzero-correction bitmap and
// correction bytes stay in its own staging slot (after the record prefix)
// until k_pack_tile writes it at its stream offset.  The slot holds a raw
// record (16 + 4 N bytes), which leaves room for all three when the rank is
// small next to n, and for the sparse entry list after them (list_cap
// entries).
struct SlotScratch {
  int64_t off_q, off_bits, off_k8, end, off_esc, esc_cap, off_list, list_cap;
  bool fits;
};
constexpr int kMaxSlotEsc = 1024;             // escapes a deferred record can carry
__host__ __device__ inline SlotScratch slot_scratch(int r, int n, int64_t L, int64_t N) {
  SlotScratch o;
  const int64_t off_pre = 16 + align_up(r, 8) + align_up((int64_t)n * r * 4, 8);   // the record's q offset
  o.off_q = align_up(off_pre, 16);
  o.off_bits = o.off_q + (int64_t)r * align_up(L, 4) * 4;
  o.off_k8 = o.off_bits + align_up(N / 8, 16);
  o.end = o.off_k8 + align_up(N, 16);
  const int64_t room = o.end <= raw_record_bytes(N, 4) ? (raw_record_bytes(N, 4) - o.end) / 4 : 0;
  o.off_esc = o.end;
  o.esc_cap = room < kMaxSlotEsc ? room / 4 * 4 : kMaxSlotEsc;
  o.off_list = o.off_esc + o.esc_cap * 4;
  o.list_cap = room - o.esc_cap;
  o.fits = r > 0 && N % 32 == 0 && N <= (int64_t)kBitsSmem * 32 && o.end <= raw_record_bytes(N, 4);
  return o;
}
constexpr int kDeferMaxWk = 7;                // deferred records have |k| < 64: no k32 values

// Record of block bi, part 1 (all threads): thread 0 works out the layout
// (raw when it is not smaller than the raw record), the block metadata and
// the column offsets.  `defer` marks a non-raw record as deferred.
__device__ void record_meta(const TileArgs& a, TileSmem& S, const Geom& g, int64_t bi, bool raw, int r, bool defer) {
  const int n = g.n;
  const int64_t L = g.L, N = g.N;
  BlockMeta& m = S.m;
  RecLayout& lay = S.lay;
  if (threadIdx.x == 0) {
    const int64_t rawsz = raw_record_bytes(N, 4);
    m.rcap = a.P.rank_cap < n ? a.P.rank_cap : n;
    m.nprobes = 0;
    for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
    m.flags = 0;
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
        m.flags |= defer ? (int)kFlagDeferred : 0;
        m.nbytes = lay.size;
      }
    }
    if (israw) {
      m.r = 0; m.wk = 0; m.ib = 0; m.ncorr = 0; m.nesc = 0;
      for (int k = 0; k < kMaxN; ++k) m.wq[k] = 0;
      m.flags = (int)kFlagRaw;
      m.nbytes = rawsz;
    }
    a.meta[bi] = m;
    if (a.ranks) a.ranks[bi] = (m.flags & kFlagRaw) ? -1 : m.r;
    int64_t wb = 0;
    for (int c = 0; c < m.r; ++c) { S.colbase[c] = wb; wb += (L * m.wq[c] + 31) / 32; }
    S.colbase[m.r] = wb;
  }
  __syncthreads();
}

// A raw record: header and the block's values in order.
__device__ void record_raw(const TileArgs& a, TileSmem& S, const Geom& g, uint8_t* rec) {
  const int tid = threadIdx.x;
  const BlockMeta& m = S.m;
  const int64_t N = g.N, M = g.M;
  if (tid == 0) {
    reinterpret_cast<uint32_t*>(rec)[0] = (uint32_t)m.flags << 8;
    reinterpret_cast<uint32_t*>(rec)[1] = 0;
    reinterpret_cast<uint32_t*>(rec)[2] = 0;
    reinterpret_cast<uint32_t*>(rec)[3] = (uint32_t)m.nbytes;
  }
  float* vals = reinterpret_cast<float*>(rec + 16);
  for (int64_t e = tid; e < N; e += kTT) {
    const int64_t lt = e / M, ls = e - lt * M;
    vals[e] = a.in[gidx_row(a, g, ls, (int)lt)];
  }
  if (tid == 0 && (16 + N * 4) % 16) {
    // zero the padding after the last value
    for (int64_t b = 16 + N * 4; b < m.nbytes; ++b) rec[b] = 0;
  }
  __syncthreads();
}

// Record prefix: padding words below `limit` zeroed, then the header, the
// column widths and the stored basis.
__device__ void record_prefix(TileSmem& S, const Geom& g, uint8_t* rec, int64_t limit) {
  const int tid = threadIdx.x, n = g.n;
  const BlockMeta& m = S.m;
  const RecLayout& lay = S.lay;
  const int rr = m.r;
  if (tid == 0) zero_padding(rec, lay, m, n, S.colbase[rr], limit);
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
  for (int c = tid; c < rr; c += kTT) rec[lay.off_wq + c] = m.wq[c];
  float* vout = reinterpret_cast<float*>(rec + lay.off_v);
  for (int i = tid; i < n * rr; i += kTT) {
    const int c = i / n, j = i - c * n;
    vout[i] = S.VstT[c * NM + j];
  }
}

// The whole record of block bi in its staging slot (k_compact moves it).
__device__ __noinline__ void write_record(const TileArgs& a, TileSmem& S, const Geom& g, int64_t bi, bool raw, int r,
                             int32_t* qs, const int8_t* k8, const int32_t* k32, const uint32_t* bits) {
  const int64_t L = g.L, N = g.N, M = g.M;
  uint8_t* rec = a.staging + align_up((g.pt_off - a.P.pt_base) * 4, 16) + 48 * bi;
  record_meta(a, S, g, bi, raw, r, false);
  const BlockMeta& m = S.m;
  const RecLayout& lay = S.lay;
  if (m.flags & kFlagRaw) {
    record_raw(a, S, g, rec);
    return;
  }
  record_prefix(S, g, rec, m.nbytes);
  pack_q(reinterpret_cast<uint32_t*>(rec + lay.off_q), qs, m.wq, S.colbase, m.r, L);
  __syncthreads();   // q scratch is free from here on
  uint32_t* cw = reinterpret_cast<uint32_t*>(rec + lay.off_c);
  if (m.wk > 0) {
    if (lay.dense) {
      // bitmap rows: k8 may hold stale bytes where the bitmap has no bit
      pack_dense(cw, k8, k32, bitmap_rows(a, g) ? bits : nullptr, m.wk, N);
    } else {
      // entry list (element indices) into the q scratch
      uint32_t* list = reinterpret_cast<uint32_t*>(qs);
      if (bitmap_rows(a, g)) {
        bitmap_list(list, bits, N, m.ncorr, S.warp_cnt);
      } else {
        compact16(
            S, k8, (int)N, [&](int8_t b, int e) { return b != 0 && (b != (int8_t)-128 || k32[e] != kEscape); },
            [&](int e, int idx) {
              if (idx < m.ncorr) list[idx] = (uint32_t)e;   // the count and the bytes agree by construction
            });
      }
      pack_sparse(cw, list, k8, k32, m.ib, m.wk, m.ncorr);
    }
  }
  if (m.nesc > 0) {
    uint32_t* ei = reinterpret_cast<uint32_t*>(rec + lay.off_ei);
    float* ev = reinterpret_cast<float*>(rec + lay.off_ev);
    compact16(
        S, k8, (int)N, [&](int8_t b, int e) { return b == (int8_t)-128 && k32[e] == kEscape; },
        [&](int e, int idx) {
          if (idx >= m.nesc) return;                      // the count and the bytes agree by construction
          ei[idx] = (uint32_t)e;
          const int64_t lt = e / M, ls = e - lt * M;
          ev[idx] = a.in[gidx_row(a, g, ls, (int)lt)];
        });
  }
  __syncthreads();
}

// A deferred record: metadata, then the prefix into the slot and the bitmap
// after the q columns; k_pack_tile does the rest once the offsets are known.
// Falls back to a raw record when the layout says so.
__device__ __noinline__ void defer_record(const TileArgs& a, TileSmem& S, const Geom& g, int64_t bi, int r,
                                          const uint32_t* bits) {
  uint8_t* slot = a.staging + align_up((g.pt_off - a.P.pt_base) * 4, 16) + 48 * bi;
  record_meta(a, S, g, bi, false, r, true);
  if (S.m.flags & kFlagRaw) {
    record_raw(a, S, g, slot);
    return;
  }
  const SlotScratch sc = slot_scratch(r, g.n, g.L, g.N);
  record_prefix(S, g, slot, sc.off_q);
  uint32_t* dst = reinterpret_cast<uint32_t*>(slot + sc.off_bits);
  for (int64_t i = threadIdx.x; i < g.N / 32; i += kTT) dst[i] = bits[i];
  __syncthreads();
}

// ---------------------------------------------------------------- the kernels
// The eigensolver out of line: inline, it would share the kernel's registers
// with the block state the body keeps live across it.
__device__ __noinline__ void jacobi_tile(TileSmem& S, int n, float jfloor) {
  if (n == NM) jacobi_cta<kTT, NM / 2>(S.G32, S.Vj, S.lam_t, n, jfloor, S.jp);
  else jacobi_cta<kTT>(S.G32, S.Vj, S.lam_t, n, jfloor, S.jp);
}

// The compression of the tile route runs as phase kernels over all its
// blocks:
//   k_gram  the Gram pass and the block statistics (streams every block once);
//   k_eig   the eigensolve, FP64 refinement, ordering and the rank prediction
//           (no staging ring: many CTAs per SM hide its barriers and its
//           FP64 latency);
//   k_enc   the encode pass at the predicted rank, the exact acceptance test
//           and the deferred record, for the blocks where all of that applies
//           (learned or tail rank, pointwise bound, full blocks);
//   k_tile  every other block, from a list k_enc fills (or all blocks with
//           the bisection): the Rayleigh-Ritz pass, the search, records that
//           cannot be deferred.  It loads the state k_gram and k_eig left, so
//           each block's basis, and so its stored bytes, do not depend on the
//           kernel that writes its record.
struct FastBlock {
  float G[NM * NM];                  // FP32 Gram, entries i, j < n
  float VstT[NM * NM];               // stored modes, VstT[k * NM + j] = Vst[j][k]
  double lam[NM];                    // eigenvalues, descending
  double lam_tr;                     // their sum
  float vsum[NM];
  float st_min[kWarps], st_max[kWarps], st_tg[kWarps], st_xg[kWarps], st_rowmax[kWarps];
  int32_t flags, rpred;
  int32_t pad[2];
};
// kFbRankFail: k_enc ran the exact test at the predicted rank and it failed
// (or a coefficient overflowed), so k_tile goes straight to the search.
enum : int32_t { kFbNonfinite = 1, kFbRR = 2, kFbOverflow = 4, kFbRankFail = 8 };

// Block counters of the phase kernels and the list of blocks k_enc leaves.
struct FastCtl {
  unsigned long long next_gram, next_eig, next_enc, next_list;
  unsigned long long nlist;
  unsigned long long next_rrg, next_rre;
  unsigned long long pad;
};

struct PhaseClock {
  long long t;
  __device__ void start() {
    if (threadIdx.x == 0) t = clock64();
  }
  __device__ void mark(TileSmem& S, int p) {
    if (threadIdx.x == 0) {
      const long long now = clock64();
      S.ph[p] += (unsigned long long)(now - t);
      t = now;
    }
  }
};

// The next block of [blo, bhi) whose Gram side is time, from a counter.
__device__ __forceinline__ int64_t grab_range(const TileArgs& a, unsigned long long* ctr) {
  for (;;) {
    const int64_t b = a.blo + (int64_t)atomicAdd(ctr, 1ull);
    if (b >= a.bhi) return a.bhi;
    if (block_geom(a.P, a.P.b0 + b).side == 0) return b;
  }
}

// Shared-memory set-up common to the kernels that stream blocks: mbarriers,
// counters and the abort flag (thread 0), then a CTA barrier.
__device__ void init_stream_smem(const TileArgs& a, TileSmem& S) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&S.full[s], a.use_tma ? 1u : (unsigned)kTT);
    mbar_init(&S.mma_bar, 1u);
    S.mma_phase = 0;
    S.mma_pending = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (threadIdx.x < kPhases) S.ph[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    S.nexact = 0;
    S.abort_flag = 0;
    S.cvar = -1;
  }
}

// Constants of the block's variable (thread 0 recomputes them when it changes).
__device__ void var_consts(TileSmem& S, const Geom& g, const VarInfo& vi, bool pointwise) {
  if (threadIdx.x == 0) {
    S.nonfinite = 0;
    S.ovf = 0;
    if (S.cvar != g.v) {
      S.cvar = g.v;
      S.crc.delta = vi.delta;
      S.crc.inv_delta = __double2float_rn(1.0 / vi.delta);
      S.crc.delta_f = __double2float_rn(vi.delta);
      S.ccc = make_corr_const(vi.eb, vi.step, pointwise);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double local_tol2(const Plan& P, const VarInfo& vi, const Geom& g) {
  return (P.eb_type == DLS_EB_NRMSE) ? (vi.eb * vi.eb) * ((double)g.N / P.kbound) : (vi.eb * vi.eb) * (double)g.N;
}

// Jacobi skip floor: rotations below 5% of the per-mode budget eb^2 L change
// no decision worth a sweep; the decisions themselves stay exact.
__device__ __forceinline__ float jacobi_floor(const TileArgs& a, const VarInfo& vi, const Geom& g, double el2) {
  return (float)(a.jfloor * (a.P.eb_type == DLS_EB_NRMSE ? el2 / g.n : vi.eb * vi.eb * (double)g.L));
}

// FP32 Jacobi, orthonormalisation of its eigenvectors, ordering, trace.
// (An FP64 Ogita-Aishima refinement step took a third of the per-block time
// and only improved eigenvector accuracy, whose effect on the energy a mode
// captures is second order; the orthonormality of the stored modes is what
// the method needs, and the re-orthonormalisation alone gives it.)
__device__ void eigen_block(TileSmem& S, int n, float jfloor, PhaseClock& pc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the eigensolve starts from the identity: its result depends on this
  // block's Gram alone, whichever blocks the CTA took before
  jacobi_tile(S, n, jfloor);
  pc.mark(S, kPhJacobi);
  orth_basis(S, n, false);
  if (warp == 0) {
    order_basis(S, n, lane);
    __syncwarp();
    if (lane == 0) {
      double tr = 0.0;
      for (int i = 0; i < n; ++i) tr += S.lam[i];
      S.lam_tr = tr;
    }
  }
  __syncthreads();
  pc.mark(S, kPhRefine);
}

// Tight bounds need the modes an FP32 Gram cannot resolve (eigenvalues near
// 2^-24 trace G): a Rayleigh-Ritz step on the projected data fixes them, when
// that resolution reaches half the per-mode budget eb^2 L.
__device__ __forceinline__ bool rr_wanted(const TileSmem& S, const Plan& P, const VarInfo& vi, const Geom& g,
                                          double el2) {
  const double budget = (vi.eb * vi.eb) * (double)g.L;
  const double noise = (P.eb_type == DLS_EB_NRMSE ? el2 / g.n : budget);
  return g.n > 1 && 4.0 * 5.9604644775390625e-8 * S.lam_tr > 0.5 * noise;
}

// |c_k| <= ||row|| (1 + 1e-4) for every column: no coefficient can reach 2^24 steps.
__device__ __forceinline__ bool overflow_possible(const TileSmem& S, const VarInfo& vi) {
  float rowmax = 0.0f;
  for (int w = 0; w < kWarps; ++w) rowmax = fmaxf(rowmax, S.st_rowmax[w]);
  return !((double)sqrtf(rowmax) * 1.0001 / vi.delta < 16777216.0 * 0.999);
}

// The predicted rank (warp 0 computes, every thread returns it).
__device__ int predicted_rank(const TileArgs& a, TileSmem& S, const Geom& g, int64_t bi, int rcap, double el2,
                              double delta) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    const int rp = predict_rank(a, S, g, bi, rcap, el2, delta, lane);
    int rm = rp;
    if (a.learned == kRankMlp && a.model) rm = mlp_rank_warp(a.model, S.featv, S.mh1, lane, rcap);
    if (lane == 0) S.r_pred = rm;
  }
  __syncthreads();
  return S.r_pred;
}

// k_gram -> state: the Gram and the statistics of the block.
__device__ void store_gram(const TileSmem& S, FastBlock& f) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NM * NM; e += kTT) f.G[e] = S.G32[e];
  if (tid < kWarps) {
    f.st_min[tid] = S.st_min[tid];
    f.st_max[tid] = S.st_max[tid];
    f.st_tg[tid] = S.st_tg[tid];
    f.st_xg[tid] = S.st_xg[tid];
    f.st_rowmax[tid] = S.st_rowmax[tid];
  }
  if (tid == 0) f.flags = S.nonfinite ? kFbNonfinite : 0;
}
// state -> k_eig: the Gram (and its FP64 copy) and the statistics.
__device__ void load_gram(TileSmem& S, const FastBlock& f, int n) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NM * NM; e += kTT) {
    const float v = f.G[e];
    S.G32[e] = v;
    if (e / NM < n && e % NM < n) S.G64[e] = (double)v;
  }
  if (tid < kWarps) {
    S.st_min[tid] = f.st_min[tid];
    S.st_max[tid] = f.st_max[tid];
    S.st_tg[tid] = f.st_tg[tid];
    S.st_xg[tid] = f.st_xg[tid];
    S.st_rowmax[tid] = f.st_rowmax[tid];
  }
  if (tid == 0) S.nonfinite = (f.flags & kFbNonfinite) ? 1 : 0;
  __syncthreads();
}
// k_eig -> state: the ordered basis, eigenvalues, flags and predicted rank.
__device__ void store_basis(const TileSmem& S, FastBlock& f, int32_t flags, int rpred) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NM * NM; e += kTT) f.VstT[e] = S.VstT[e];
  if (tid < NM) {
    f.vsum[tid] = S.vsum[tid];
    f.lam[tid] = S.lam[tid];
  }
  if (tid == 0) {
    f.lam_tr = S.lam_tr;
    f.flags = flags;
    f.rpred = rpred;
  }
}
// state -> k_enc / k_tile: everything the passes after the eigensolve read.
__device__ void load_basis(TileSmem& S, const FastBlock& f) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NM * NM; e += kTT) S.VstT[e] = f.VstT[e];
  if (tid < NM) {
    S.vsum[tid] = f.vsum[tid];
    S.lam[tid] = f.lam[tid];
  }
  if (tid < kWarps) {
    S.st_min[tid] = f.st_min[tid];
    S.st_max[tid] = f.st_max[tid];
    S.st_tg[tid] = f.st_tg[tid];
    S.st_xg[tid] = f.st_xg[tid];
    S.st_rowmax[tid] = f.st_rowmax[tid];
  }
  if (tid == 0) {
    S.lam_tr = f.lam_tr;
    S.nonfinite = (f.flags & kFbNonfinite) ? 1 : 0;
    S.r_pred = f.rpred;
  }
  __syncthreads();
}

// Phase counters of a phase kernel's CTA into the workspace slot it shares
// with others (more CTAs than slots).
__device__ void flush_phases(const TileArgs& a, TileSmem& S) {
  if (threadIdx.x == 0) {
    S.ph[kCntExact] += S.nexact;
    if (a.phase)
      for (int i = 0; i < kPhases; ++i)
        if (S.ph[i]) atomicAdd(&a.phase[(int64_t)(blockIdx.x % a.ctas) * kPhases + i], S.ph[i]);
  }
}

// Leaves no copy and no product in flight, then gives back the TMEM.
template <bool TC>
__device__ void finish_stream(TileSmem& S, Cursor& cu) {
  while (cu.con < cu.iss) {
    mbar_wait(&S.full[cu.con % kStages], (cu.con / kStages) & 1u);
    ++cu.con;
  }
  if (TC) {
    if (threadIdx.x == 0 && S.mma_pending) mbar_wait(&S.mma_bar, S.mma_phase & 1u);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                   : "memory");
    }
  }
}

template <bool TC>
__device__ void alloc_tmem(TileSmem& S) {
  if (TC) {
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                   "r"(kTmemCols)
                   : "memory");
      // give up the allocation permit at once, so further CTAs can become resident
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ TileSmem& tile_smem(unsigned char* smem_raw) {
  // TMA destinations: align the tile ring to 1024 bytes explicitly
  const uint32_t sbase = smem_u32(smem_raw);
  return *reinterpret_cast<TileSmem*>(smem_raw + (((sbase + 1023u) & ~1023u) - sbase));
}

// ---------------------------------------------------------------- k_gram
// The Gram pass of every block of the launch's range: FP32 Gram (or the
// 3xTF32 tensor-core Gram) and statistics into the block's state.
template <int MINB, bool TC>
__global__ void __launch_bounds__(kTT, MINB) k_gram(const __grid_constant__ CUtensorMap tmap,
                                                    const __grid_constant__ CUtensorMap tmapg,
                                                    const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = tile_smem(smem_raw);
  const Maps tm{&tmap, &tmapg};
  const Plan& P = a.P;
  float* lobuf = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(&S) +
                                          align_up((int64_t)sizeof(TileSmem), 1024));
  (void)lobuf;
  init_stream_smem(a, S);
  alloc_tmem<TC>(S);
  PhaseClock pc;
  Cursor cu;
  cu.iss = 0; cu.con = 0; cu.pf_blk = -1; cu.pf_cnt = 0; cu.pf_layout = kLayoutRow;
  if (threadIdx.x == 0) S.bnext = grab_range(a, &a.ctl->next_gram);
  __syncthreads();
  for (;;) {
    const int64_t bi = S.bnext;
    __syncthreads();
    if (bi >= a.bhi) break;
    if (threadIdx.x == 0) S.bnext = grab_range(a, &a.ctl->next_gram);
    const Geom g = block_geom(P, P.b0 + bi);
    if (threadIdx.x == 0) S.nonfinite = 0;
    __syncthreads();
    pc.start();
    bool ok;
    if (TC) ok = pass_gram_tc(a, tm, S, cu, bi, g, lobuf);
    else ok = g.n == NM ? pass_gram<false, NM>(a, tm, S, cu, bi, g) : pass_gram<false, 0>(a, tm, S, cu, bi, g);
    if (!ok) break;
    // the next block's first chunks load while this one's state is written
    {
      const int64_t bn = S.bnext;
      if (bn < a.bhi) prefetch(a, tm, S, cu, bn, block_geom(P, P.b0 + bn), TC ? kLayoutGram : kLayoutRow);
    }
    if (S.nonfinite && threadIdx.x == 0) atomicOr(&a.status->nonfinite, 1u);
    store_gram(S, a.fb[bi]);
    pc.mark(S, kPhGram);
    __syncthreads();
  }
  if (S.abort_flag && threadIdx.x == 0) atomicOr(&a.status->timeout, 1u);
  finish_stream<TC>(S, cu);
  flush_phases(a, S);
}

// The next block of the range that k_eig flagged for the Rayleigh-Ritz pass.
__device__ __forceinline__ int64_t grab_rr(const TileArgs& a, unsigned long long* ctr) {
  for (;;) {
    const int64_t b = grab_range(a, ctr);
    if (b >= a.bhi || (a.fb[b].flags & kFbRR)) return b;
  }
}

// ---------------------------------------------------------------- k_eig
// Eigensolve, orthonormalisation, ordering and rank prediction of every block
// of the range, from the Gram k_gram left.  Blocks whose FP32 Gram cannot
// resolve the modes near the budget are flagged for the Rayleigh-Ritz pass,
// blocks whose coefficients might overflow for k_tile.
// RR: the second solve of the Rayleigh-Ritz pass, on the flagged blocks, from
// the Gram of their rows projected on the first basis (k_rrgram): the rotated
// basis V = Vst W in FP64, orthonormalised, ordered, and the rank predicted.
template <bool RR>
// Twelve CTAs per SM (40 registers, 18 KB of shared memory each): the CTA
// Jacobi waits at a barrier after every round, and more resident CTAs hide it
// (16384 blocks of order 16: 0.95 ms at 5 CTAs per SM, 0.79 at 8, 0.69 at 12).
__global__ void __launch_bounds__(kTT, 12) k_eig(const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = tile_smem(smem_raw);       // only the part before the staging ring
  const Plan& P = a.P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long* ctr = RR ? &a.ctl->next_rre : &a.ctl->next_eig;
  auto next = [&]() { return RR ? grab_rr(a, ctr) : grab_range(a, ctr); };
  if (tid < kPhases) S.ph[tid] = 0;
  if (tid == 0) {
    S.nexact = 0;
    S.bnext = next();
  }
  __syncthreads();
  PhaseClock pc;
  for (;;) {
    const int64_t bi = S.bnext;
    __syncthreads();
    if (bi >= a.bhi) break;
    if (tid == 0) S.bnext = next();
    const Geom g = block_geom(P, P.b0 + bi);
    const VarInfo vi = a.vars[g.v];
    const int n = g.n;
    const int rcap = P.rank_cap < n ? P.rank_cap : n;
    const double el2 = local_tol2(P, vi, g);
    FastBlock& f = a.fb[bi];
    pc.start();
    const int32_t flags0 = f.flags;
    load_gram(S, f, n);
    if (S.nonfinite) continue;                  // k_gram has set the status
    const float jfloor = jacobi_floor(a, vi, g, el2);
    int32_t flags = 0;
    if (RR) {
      load_basis(S, f);                         // the first basis
      jacobi_tile(S, n, jfloor);
      // V = Vst W, orthonormalised; eigenvalues from the Rayleigh-Ritz diagonal
      orth_basis(S, n, true);
      if (warp == 0) order_basis(S, n, lane);
      __syncthreads();
      pc.mark(S, kPhRR);
      flags = flags0 & ~kFbRR;
    } else {
      eigen_block(S, n, jfloor, pc);
      if (rr_wanted(S, P, vi, g, el2)) flags |= kFbRR;
      if (overflow_possible(S, vi)) flags |= kFbOverflow;
    }
    int rp = 0;
    if (!(flags & kFbRR)) rp = predicted_rank(a, S, g, bi, rcap, el2, vi.delta);
    pc.mark(S, kPhPredict);
    store_basis(S, f, flags, rp);
    __syncthreads();
  }
  flush_phases(a, S);
}

// ---------------------------------------------------------------- k_rrgram
// First half of the Rayleigh-Ritz pass, for the blocks k_eig flagged: the Gram
// of the block's rows projected on its first basis (the coefficients the
// encode pass computes), into the block's state for k_eig<true>.
template <int MINB>
__global__ void __launch_bounds__(kTT, MINB) k_rrgram(const __grid_constant__ CUtensorMap tmap,
                                                      const __grid_constant__ CUtensorMap tmapg,
                                                      const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = tile_smem(smem_raw);
  const Maps tm{&tmap, &tmapg};
  const Plan& P = a.P;
  init_stream_smem(a, S);
  __syncthreads();
  PhaseClock pc;
  Cursor cu;
  cu.iss = 0; cu.con = 0; cu.pf_blk = -1; cu.pf_cnt = 0; cu.pf_layout = kLayoutRow;
  if (threadIdx.x == 0) S.bnext = grab_rr(a, &a.ctl->next_rrg);
  __syncthreads();
  for (;;) {
    const int64_t bi = S.bnext;
    __syncthreads();
    if (bi >= a.bhi) break;
    if (threadIdx.x == 0) S.bnext = grab_rr(a, &a.ctl->next_rrg);
    const Geom g = block_geom(P, P.b0 + bi);
    pc.start();
    load_basis(S, a.fb[bi]);
    const bool ok = g.n == NM ? pass_gram<true, NM>(a, tm, S, cu, bi, g) : pass_gram<true, 0>(a, tm, S, cu, bi, g);
    if (!ok) break;
    {
      const int64_t bn = S.bnext;
      if (bn < a.bhi) prefetch(a, tm, S, cu, bn, block_geom(P, P.b0 + bn), kLayoutRow);
    }
    FastBlock& f = a.fb[bi];
    for (int e = threadIdx.x; e < NM * NM; e += kTT) f.G[e] = S.G32[e];
    pc.mark(S, kPhRR);
    __syncthreads();
  }
  if (S.abort_flag && threadIdx.x == 0) atomicOr(&a.status->timeout, 1u);
  finish_stream<false>(S, cu);
  flush_phases(a, S);
}

// ---------------------------------------------------------------- k_enc
// Encode pass at the predicted rank, exact acceptance test (pass(r) and not
// pass(r - 1), FP64 semantics) and the deferred record, for the blocks where
// all of that applies; every other block goes to the list k_tile takes.
template <int MINB>
__global__ void __launch_bounds__(kTT, MINB) k_enc(const __grid_constant__ CUtensorMap tmap,
                                                   const __grid_constant__ CUtensorMap tmapg,
                                                   const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = tile_smem(smem_raw);
  const Maps tm{&tmap, &tmapg};
  const Plan& P = a.P;
  int32_t* k32 = a.k32_scr + (int64_t)blockIdx.x * a.nptmax;
  init_stream_smem(a, S);
  __syncthreads();
  PhaseClock pc;
  Cursor cu;
  cu.iss = 0; cu.con = 0; cu.pf_blk = -1; cu.pf_cnt = 0; cu.pf_layout = kLayoutRow;
  auto eligible = [&](int64_t b, int* rp_out) -> bool {
    const Geom gb = block_geom(P, P.b0 + b);
    const FastBlock& fb = a.fb[b];
    const int rp = fb.rpred;
    *rp_out = rp;
    return !(fb.flags & (kFbNonfinite | kFbRR | kFbOverflow)) && gb.n == NM && bitmap_rows(a, gb) &&
           gb.N <= (int64_t)kBitsSmem * 32 && slot_scratch(rp, gb.n, gb.L, gb.N).fits;
  };
  auto to_list = [&](int64_t b) {
    if (threadIdx.x == 0) {
      const unsigned long long i = atomicAdd(&a.ctl->nlist, 1ull);
      a.list[i] = (int32_t)b;
    }
  };
  const bool pointwise = P.eb_type != DLS_EB_NRMSE;
  if (threadIdx.x == 0) S.bnext = grab_range(a, &a.ctl->next_enc);
  __syncthreads();
  for (;;) {
    const int64_t bi = S.bnext;
    __syncthreads();
    if (bi >= a.bhi) break;
    if (threadIdx.x == 0) S.bnext = grab_range(a, &a.ctl->next_enc);
    const Geom g = block_geom(P, P.b0 + bi);
    int rp = 0;
    if (!pointwise || !eligible(bi, &rp)) {
      if (!(a.fb[bi].flags & kFbNonfinite)) to_list(bi);
      __syncthreads();          // thread 0 has taken the next block
      continue;
    }
    const VarInfo vi = a.vars[g.v];
    const double el2 = local_tol2(P, vi, g);
    var_consts(S, g, vi, pointwise);
    const RowConst rcst = S.crc;
    const CorrConst cc = S.ccc;
    pc.start();
    load_basis(S, a.fb[bi]);
    uint8_t* const slot = a.staging + align_up((g.pt_off - P.pt_base) * 4, 16) + 48 * bi;
    const SlotScratch sc = slot_scratch(rp, g.n, g.L, g.N);
    if (threadIdx.x == 0) {
      S.esc_list = reinterpret_cast<uint32_t*>(slot + sc.off_esc);
      S.esc_cap = (int)sc.esc_cap;
    }
    if (!pass_encode<NM, true>(a, tm, S, cu, bi, g, rp, true, rcst, cc, true,
                               reinterpret_cast<int32_t*>(slot + sc.off_q), reinterpret_cast<int8_t*>(slot + sc.off_k8),
                               k32, S.bitsm))
      break;
    pc.mark(S, kPhEncode);
    bool accepted = false;
    if (!S.ovf) {
      const Chunks chk = chunks_of(a, g);
      const double bnd = (double)(cdiv(a.rc, kTT) * chk.n * g.n + 40) * 6.6e-8;
      const double E_rm1 = S.Ered[0], E_r = S.Ered[1];
      const bool p_r = decide_pass(a, S, g, rp, E_r, bnd, el2, rcst);
      bool p_rm1 = false;
      if (rp > 0 && p_r) p_rm1 = decide_pass(a, S, g, rp - 1, E_rm1, bnd, el2, rcst);
      accepted = p_r && !p_rm1;
    }
    // k_tile would repeat this very test (same pass, same inputs, same
    // decision) before searching: record that it failed
    const bool rank_fail = !accepted;
    // a deferred record has no correction beyond kDeferMaxWk bits, its
    // escapes fit the slot's list and, when sparse, so does its entry list
    if (accepted) {
      const int wk = bit_width((uint32_t)S.kmax), ib = bit_width((uint32_t)(g.N - 1));
      const bool dense = wk > 0 && (g.N * wk + 31) / 32 < ((int64_t)S.ncorr * (ib + wk) + 31) / 32;
      if (wk > kDeferMaxWk || (!dense && S.ncorr > sc.list_cap) || S.nesc > sc.esc_cap) accepted = false;
    }
    pc.mark(S, kPhDecide);
    if (!accepted) {
      if (rank_fail && threadIdx.x == 0) a.fb[bi].flags |= kFbRankFail;
      to_list(bi);
      __syncthreads();
      continue;
    }
    {
      int rn = 0;
      const int64_t bn = S.bnext;
      if (bn < a.bhi && pointwise && eligible(bn, &rn)) prefetch(a, tm, S, cu, bn, block_geom(P, P.b0 + bn), kLayoutRow);
    }
    defer_record(a, S, g, bi, rp, S.bitsm);
    pc.mark(S, kPhPack);
    if (threadIdx.x == 0) S.ph[kCntAccepted] += 1;
  }
  if (S.abort_flag && threadIdx.x == 0) atomicOr(&a.status->timeout, 1u);
  finish_stream<false>(S, cu);
  flush_phases(a, S);
}

// ---------------------------------------------------------------- k_tile
// Every block k_enc does not finish, with the block state (basis, eigenvalues,
// statistics) k_gram and k_eig left: the Rayleigh-Ritz pass where the FP32
// Gram cannot resolve the modes near the budget, the rank test of a
// prediction and the bisection of Algorithm 1 when it fails (or always, with
// the search rank mode), and records that cannot be deferred.  With
// a.from_list the blocks come from k_enc's list, else from the launch range.
// The arguments stay in parameter space (the passes take their address).
template <int MINB>
__global__ void __launch_bounds__(kTT, MINB) k_tile(const __grid_constant__ CUtensorMap tmap,
                                                    const __grid_constant__ CUtensorMap tmapg,
                                                    const __grid_constant__ TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem& S = tile_smem(smem_raw);
  const Maps tm{&tmap, &tmapg};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* qs = a.q_scr + (int64_t)blockIdx.x * NM * a.lmax;
  int8_t* k8 = a.k8_scr + (int64_t)blockIdx.x * a.nptmax;
  int32_t* k32 = a.k32_scr + (int64_t)blockIdx.x * a.nptmax;
  uint32_t* bits = a.bit_scr + (int64_t)blockIdx.x * (align_up(a.nptmax, 32) / 32);
  const Plan& P = a.P;
  init_stream_smem(a, S);
  __syncthreads();
  PhaseClock pc;
  // blocks whose Gram side is time; the others are left to k_mixed
  auto grab = [&]() -> int64_t {
    if (a.from_list) {
      const unsigned long long i = atomicAdd(&a.ctl->next_list, 1ull);
      return i < a.ctl->nlist ? (int64_t)a.list[i] : a.bhi;
    }
    return grab_range(a, &a.status->pad[1]);
  };
  Cursor cu;
  cu.iss = 0; cu.con = 0; cu.pf_blk = -1; cu.pf_cnt = 0; cu.pf_layout = kLayoutRow;
  if (tid == 0) S.bnext = grab();
  __syncthreads();
  for (;;) {
    const int64_t bi = S.bnext;
    __syncthreads();
    if (bi >= a.bhi) break;
    if (tid == 0) S.bnext = grab();
    const Geom g = block_geom(P, P.b0 + bi);
    const VarInfo vi = a.vars[g.v];
    const int n = g.n;
    const int rcap = P.rank_cap < n ? P.rank_cap : n;
    const bool pointwise = P.eb_type != DLS_EB_NRMSE;
    const double el2 = local_tol2(P, vi, g);
    var_consts(S, g, vi, pointwise);
    const RowConst rcst = S.crc;
    const CorrConst cc = S.ccc;

    pc.start();
    const bool full = n == NM;   // Gram order 16: the passes without per-column predicates
    const float jfloor = jacobi_floor(a, vi, g, el2);
    load_basis(S, a.fb[bi]);
    if (S.nonfinite) continue;                  // k_gram has set the status
    prefetch(a, tm, S, cu, bi, g, kLayoutRow);
    // the Rayleigh-Ritz pass, if k_rrgram and k_eig<true> have not done it
    bool did_rr = false;
    if (a.fb[bi].flags & kFbRR) {
      did_rr = true;
      if (!(full ? pass_gram<true, NM>(a, tm, S, cu, bi, g) : pass_gram<true, 0>(a, tm, S, cu, bi, g))) break;
      prefetch(a, tm, S, cu, bi, g, kLayoutRow);
      jacobi_tile(S, n, jfloor);
      // V = Vst W, orthonormalised; eigenvalues from the Rayleigh-Ritz diagonal
      orth_basis(S, n, true);
      if (warp == 0) order_basis(S, n, lane);
      __syncthreads();
    }
    pc.mark(S, kPhRR);

    const bool may_overflow = overflow_possible(S, vi);
    // the prediction k_eig made, unless the Rayleigh-Ritz pass changed the basis
    if (did_rr) predicted_rank(a, S, g, bi, rcap, el2, vi.delta);
    pc.mark(S, kPhPredict);

    // the encode pass at rank rr; SPARSE where the bitmap carries the corrections,
    // kept in shared memory when the block has at most kBitsSmem * 32 points
    const bool sparse = pointwise && bitmap_rows(a, g);
    uint32_t* const bitp = g.N <= (int64_t)kBitsSmem * 32 ? S.bitsm : bits;
    // SPARSE passes whose rank leaves room write q and k8 into the block's
    // staging slot (deferred packing); the others use the CTA's scratch
    uint8_t* const slot = a.staging + align_up((g.pt_off - P.pt_base) * 4, 16) + 48 * bi;
    bool in_slot = false;
    auto encode = [&](int rr, bool check, bool sp, bool cta_scratch) -> bool {
      in_slot = false;
      if (sp) {
        int32_t* q = qs;
        int8_t* k = k8;
        uint32_t* esc = nullptr;
        const SlotScratch sc = slot_scratch(rr, g.n, g.L, g.N);
        if (!cta_scratch && sc.fits) {
          q = reinterpret_cast<int32_t*>(slot + sc.off_q);
          k = reinterpret_cast<int8_t*>(slot + sc.off_k8);
          esc = reinterpret_cast<uint32_t*>(slot + sc.off_esc);
          in_slot = true;
        }
        if (tid == 0) { S.esc_list = esc; S.esc_cap = (int)sc.esc_cap; }   // read after the pass's first barrier
        return full ? pass_encode<NM, true>(a, tm, S, cu, bi, g, rr, check, rcst, cc, pointwise, q, k, k32, bitp)
                    : pass_encode<0, true>(a, tm, S, cu, bi, g, rr, check, rcst, cc, pointwise, q, k, k32, bitp);
      }
      if (tid == 0) S.esc_list = nullptr;
      return full ? pass_encode<NM, false>(a, tm, S, cu, bi, g, rr, check, rcst, cc, pointwise, qs, k8, k32, bitp)
                  : pass_encode<0, false>(a, tm, S, cu, bi, g, rr, check, rcst, cc, pointwise, qs, k8, k32, bitp);
    };
    const Chunks chk = chunks_of(a, g);
    const int64_t rows_per_thread = cdiv(a.rc, kTT) * chk.n;
    const double bnd = (double)(rows_per_thread * n + 40) * 6.6e-8;
    bool accepted = false;
    int r = 0;
    if (a.learned != kRankSearch && !may_overflow && !(a.fb[bi].flags & kFbRankFail)) {
      const int rp = S.r_pred;
      if (!encode(rp, true, sparse, false)) break;
      pc.mark(S, kPhEncode);
      const double E_rm1 = S.Ered[0], E_r = S.Ered[1];
      if (!S.ovf) {
        const bool p_r = decide_pass(a, S, g, rp, E_r, bnd, el2, rcst);
        bool p_rm1 = false;
        if (rp > 0 && p_r) p_rm1 = decide_pass(a, S, g, rp - 1, E_rm1, bnd, el2, rcst);
        accepted = p_r && !p_rm1;
        r = rp;
      }
      pc.mark(S, kPhDecide);
    }
    bool raw = false;
    if (!accepted) {
      // every warp has read S.ovf (above) before thread 0 clears it: a warp
      // that read the cleared flag would take the decision the others skip,
      // and the CTA's barriers and chunk arrivals would no longer pair up
      __syncthreads();
      if (tid == 0) S.ovf = 0;
      __syncthreads();
      int ovf = 0;
      if (!(full ? pass_all_errors<NM>(a, tm, S, cu, bi, g, rcap, rcst, ovf)
                 : pass_all_errors<0>(a, tm, S, cu, bi, g, rcap, rcst, ovf)))
        break;
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
          if (decide_pass(a, S, g, mid, Eall[mid], bnd, el2, rcst)) hi = mid;
          else lo = mid + 1;
        }
        r = lo;
        if (!pointwise && !decide_pass(a, S, g, r, Eall[r], bnd, el2, rcst)) raw = true;
        if (!raw && !encode(r, false, sparse, false)) break;
      }
      pc.mark(S, kPhSearch);
    }
    // a deferred record has no correction beyond kDeferMaxWk bits, its
    // escapes fit the slot's list and, when sparse, so does its entry list;
    // otherwise the block is encoded again into the CTA's scratch for the
    // record writer here, with every element written when it has escapes
    // (the writer lists escapes from k8 itself)
    // (the pass's counters are read into registers, and a barrier passed,
    // before another pass lets thread 0 reset them)
    if (!raw && in_slot) {
      // the layout's own choice: a dense record needs no entry list
      const int kmax = S.kmax, ncorr = S.ncorr, nesc = S.nesc;
      const int wk = bit_width((uint32_t)kmax), ib = bit_width((uint32_t)(g.N - 1));
      const bool dense = wk > 0 && (g.N * wk + 31) / 32 < ((int64_t)ncorr * (ib + wk) + 31) / 32;
      const SlotScratch sc = slot_scratch(r, g.n, g.L, g.N);
      __syncthreads();
      if (wk > kDeferMaxWk || (!dense && ncorr > sc.list_cap) || nesc > sc.esc_cap)
        if (!encode(r, false, nesc == 0, true)) break;
    } else if (!raw && sparse) {
      const int nesc = S.nesc;
      __syncthreads();
      if (nesc > 0 && !encode(r, false, false, true)) break;
    }
    const bool deferred = !raw && in_slot;
    // the next block's first chunks load while this record is packed
    {
      const int64_t bn = S.bnext;
      if (bn < a.bhi) prefetch(a, tm, S, cu, bn, block_geom(P, P.b0 + bn), kLayoutRow);
    }
    if (deferred) defer_record(a, S, g, bi, r, bitp);
    else write_record(a, S, g, bi, raw, r, qs, k8, k32, bitp);
    pc.mark(S, kPhPack);
    if (tid == 0) S.ph[accepted ? kCntAccepted : kCntSearched] += 1;
  }
  if (S.abort_flag) {
    if (tid == 0) atomicOr(&a.status->timeout, 1u);
  }
  finish_stream<false>(S, cu);
  if (tid == 0) {
    S.ph[kCntExact] = S.nexact;
    if (a.phase)
      for (int i = 0; i < kPhases; ++i) a.phase[(int64_t)blockIdx.x * kPhases + i] += S.ph[i];
  }
}

// ---------------------------------------------------------------- deferred packing
// Packs the records the tile kernel left in their staging slots, straight to
// their stream offsets (after the scan).  One CTA per block at a time, many
// CTAs per SM: the bit packing is short dependent chains, which a full SM of
// warps overlaps.
__global__ void __launch_bounds__(kTT, 6) k_pack_tile(Plan P, const BlockMeta* meta, uint8_t* staging,
                                                      const unsigned long long* offsets, Status* st, uint8_t* out,
                                                      const float* in) {
  __shared__ BlockMeta m;
  __shared__ RecLayout lay;
  __shared__ int64_t colbase[NM + 1];
  __shared__ int warp_cnt[kWarps];
  __shared__ __align__(16) uint32_t bitsm[kBitsSmem];
  __shared__ uint32_t esc_in[kMaxSlotEsc], esc_sorted[kMaxSlotEsc];
  __shared__ int skip;
  if (st->capacity || st->nonfinite || st->timeout) return;
  const int tid = threadIdx.x;
  for (int64_t bi = blockIdx.x; bi < P.nb; bi += gridDim.x) {
    const Geom g = block_geom(P, P.b0 + bi);
    if (tid == 0) {
      m = meta[bi];
      int sk = !(m.flags & kFlagDeferred);
      if (!sk) {
        lay = rec_layout(m.r, g.n, g.L, g.N, 4, m.wq, m.wk, m.ib, m.ncorr, m.nesc);
        const SlotScratch sc = slot_scratch(m.r, g.n, g.L, g.N);
        // a deferred record is one the tile kernel could defer: check before use
        if (!sc.fits || lay.size != m.nbytes || m.nesc > sc.esc_cap || m.wk > kDeferMaxWk || m.r > g.n ||
            (!lay.dense && m.ncorr > sc.list_cap)) {
          atomicOr(&st->corrupt, 1u);
          sk = 1;
        }
        int64_t wb = 0;
        for (int c = 0; c < m.r && c < NM; ++c) { colbase[c] = wb; wb += (g.L * m.wq[c] + 31) / 32; }
        colbase[m.r < NM ? m.r : NM] = wb;
      }
      skip = sk;
    }
    __syncthreads();
    if (skip) {
      __syncthreads();
      continue;
    }
    const SlotScratch sc = slot_scratch(m.r, g.n, g.L, g.N);
    uint8_t* slot = staging + align_up((g.pt_off - P.pt_base) * 4, 16) + 48 * bi;
    uint8_t* rec = out + P.payload_pos + offsets[bi];
    if (tid == 0) zero_padding(rec, lay, m, g.n, colbase[m.r], m.nbytes);
    __syncthreads();
    // the prefix (header, widths, basis; its padding zeroed) as it is
    for (int64_t i = tid; i < lay.off_q / 8; i += kTT)
      reinterpret_cast<uint2*>(rec)[i] = reinterpret_cast<const uint2*>(slot)[i];
    const int64_t nw = g.N / 32;
    for (int64_t i = tid; i < nw; i += kTT) bitsm[i] = reinterpret_cast<const uint32_t*>(slot + sc.off_bits)[i];
    const int32_t* qs = reinterpret_cast<const int32_t*>(slot + sc.off_q);
    const int8_t* k8 = reinterpret_cast<const int8_t*>(slot + sc.off_k8);
    pack_q<true>(reinterpret_cast<uint32_t*>(rec + lay.off_q), qs, m.wq, colbase, m.r, g.L);
    __syncthreads();
    if (m.wk > 0) {
      uint32_t* cw = reinterpret_cast<uint32_t*>(rec + lay.off_c);
      if (lay.dense) {
        pack_dense<true>(cw, k8, nullptr, bitsm, m.wk, g.N);
      } else {
        uint32_t* list = reinterpret_cast<uint32_t*>(slot + sc.off_list);
        bitmap_list(list, bitsm, g.N, m.ncorr, warp_cnt);
        pack_sparse<true>(cw, list, k8, nullptr, m.ib, m.wk, m.ncorr);
      }
    }
    if (m.nesc > 0) {
      // escapes were listed in no particular order: each goes to its rank
      // among them (element order, the indices being distinct)
      const int ne = m.nesc;
      const uint32_t* el = reinterpret_cast<const uint32_t*>(slot + sc.off_esc);
      for (int i = tid; i < ne; i += kTT) esc_in[i] = el[i];
      __syncthreads();
      for (int i = tid; i < ne; i += kTT) {
        const uint32_t e = esc_in[i];
        int rank = 0;
        for (int j = 0; j < ne; ++j) rank += esc_in[j] < e ? 1 : 0;
        esc_sorted[rank] = e;
      }
      __syncthreads();
      uint32_t* ei = reinterpret_cast<uint32_t*>(rec + lay.off_ei);
      float* ev = reinterpret_cast<float*>(rec + lay.off_ev);
      for (int i = tid; i < ne; i += kTT) {
        const uint32_t e = esc_sorted[i];
        const int64_t lt = e / g.M, ls = e - lt * g.M;
        ei[i] = e;
        ev[i] = in[gidx_plan(P, g, ls, (int)lt)];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

}  // namespace

// Chunk box of the plan: (bxb, yc, zc, bt) with bxb * yc * zc * bt <= one stage.
bool tile_chunk_box(const Plan& p, int* bxb, int* yc, int* zc, int* bt) {
  const int bx = p.block[0], by = p.block[1], bz = p.block[2], btt = p.block[3];
  if (btt > NM || bx * btt > kStageFloats) return false;
  *bxb = bx;
  *bt = btt;
  if (bx * by * btt <= kStageFloats) {
    *yc = by;
    const int z = kStageFloats / (bx * by * btt);
    *zc = z < bz ? z : bz;
  } else {
    *yc = kStageFloats / (bx * btt);
    *zc = 1;
  }
  return true;
}

int64_t pitched_row(const Plan& p, bool staged) {
  if (!staged || p.dtype != DLS_F32 || p.b0 != 0 || p.nb != p.nb_total || p.nb == 0) return 0;
  if (p.dims[0] % 4 == 0 || p.block[0] % 4 != 0) return 0;
  return align_up(p.dims[0], 4);
}

// The pitched copy: one warp per x line (rows = nvars * nt * nz * ny), the
// line's nx values then zeros up to the pitch.  Pairs of floats where nx is
// even and the input 8-byte aligned (the copy's lines start on 16 bytes).
__global__ void __launch_bounds__(256) k_pitch_rows(const float* __restrict__ in, float* __restrict__ out,
                                                    int64_t rows, int64_t nx, int64_t pitch, int pairs) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw) {
    const float* src = in + r * nx;
    float* dst = out + r * pitch;
    if (pairs) {
      const float2* s2 = reinterpret_cast<const float2*>(src);
      float2* d2 = reinterpret_cast<float2*>(dst);
      for (int64_t i = lane; i < nx / 2; i += 32) d2[i] = __ldg(s2 + i);
    } else {
      for (int64_t i = lane; i < nx; i += 32) dst[i] = __ldg(src + i);
    }
    for (int64_t i = nx + lane; i < pitch; i += 32) dst[i] = 0.0f;
  }
}

// Dynamic shared memory: alignment slack, the shared struct, and with the
// tensor-core Gram the 16 KiB lo buffer.
size_t tile_smem_bytes(bool tc) {
  return 1024 + (size_t)align_up((int64_t)sizeof(TileSmem), 1024) + (tc ? (size_t)kStageFloats * 4 : 0);
}

// Dynamic shared memory of k_eig: the shared struct up to the staging ring.
size_t eig_smem_bytes() { return 1024 + (size_t)offsetof(TileSmem, ring); }

// Resident CTAs per SM from the kernel's registers and shared memory and the
// device's per-SM limits (and, with the tensor-core Gram, the TMEM columns).
// Computed here because the occupancy query treats a kernel that contains
// tcgen05.alloc as one CTA per SM.
template <class K>
int ctas_per_sm_of(K kernel, size_t smem, bool tc) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaFuncAttributes fa;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return 0;
  // registers are allocated per warp in units of 256
  const int regs_warp = (int)align_up((int64_t)fa.numRegs * 32, 256);
  const int by_regs = prop.regsPerMultiprocessor / (regs_warp * (kTT / 32));
  const int by_smem = (int)(prop.sharedMemPerMultiprocessor /
                            (smem + (size_t)fa.sharedSizeBytes + prop.reservedSharedMemPerBlock));
  const int by_threads = prop.maxThreadsPerMultiProcessor / kTT;
  int n = by_regs < by_smem ? by_regs : by_smem;
  n = n < by_threads ? n : by_threads;
  n = n < prop.maxBlocksPerMultiProcessor ? n : prop.maxBlocksPerMultiProcessor;
  if (tc) n = n < (int)(512 / kTmemCols) ? n : (int)(512 / kTmemCols);
  return n;
}

int tile_ctas_per_sm(int variant) {
  const size_t sm = tile_smem_bytes(false);
  const int n = variant == 1 ? ctas_per_sm_of(k_tile<2>, sm, false) : ctas_per_sm_of(k_tile<4>, sm, false);
  cudaGetLastError();
  return n;
}

// Bytes of the phase kernels' state in the workspace for a plan of nb blocks.
size_t tile_fast_bytes(int64_t nb) {
  const int64_t n1 = nb > 0 ? nb : 1;
  return (size_t)align_up((int64_t)sizeof(FastCtl), 256) + (size_t)align_up(n1 * (int64_t)sizeof(FastBlock), 256) +
         (size_t)align_up(n1 * 4, 256);
}

int launch_tile_compress(const Plan& p, const void* d_in, const MixedWork& w, int learned, Occupancy occ,
                         cudaStream_t s, int64_t blo, int64_t bhi, const cudaEvent_t* pev) {
  auto mark = [&](int i) -> bool {
    return !pev || !pev[i] || record_marker(pev[i], s) == cudaSuccess;
  };
  if (bhi < 0) bhi = p.nb;
  if (blo < 0 || blo > bhi || bhi > p.nb || !w.fast || !w.phase || w.ctas < 1) return DLS_ERR_INVALID_ARG;
  if (bhi == blo) return DLS_OK;
  TileArgs a;
  memset(&a, 0, sizeof(a));
  a.P = p;
  a.blo = blo;
  a.bhi = bhi;
  a.in = (const float*)d_in;
  a.staging = w.staging;
  a.meta = w.meta;
  a.vars = w.vars;
  a.status = w.status;
  a.q_scr = w.q_scr;
  a.k8_scr = w.k8_scr;
  a.k32_scr = w.k32_scr;
  a.bit_scr = w.bit_scr;
  a.feat = w.feat;
  a.ranks = w.ranks;
  a.lmax = w.lmax;
  a.nptmax = w.nptmax;
  a.learned = learned;
  a.phase = w.phase;
  a.withhold = fault_withheld_block();
  a.model = rank_model_device();
  a.ctas = w.ctas;
  {
    uint8_t* f = w.fast;
    a.ctl = reinterpret_cast<FastCtl*>(f);
    f += align_up((int64_t)sizeof(FastCtl), 256);
    a.fb = reinterpret_cast<FastBlock*>(f);
    f += align_up((p.nb > 0 ? p.nb : 1) * (int64_t)sizeof(FastBlock), 256);
    a.list = reinterpret_cast<int32_t*>(f);
  }
  if (!tile_chunk_box(p, &a.bxb, &a.yc, &a.zc, &a.bt)) return DLS_ERR_INVALID_ARG;
  a.rc = a.bxb * a.yc * a.zc;
  auto magic = [](int d) -> uint32_t { return d <= 1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)d - 1) / (uint64_t)d); };
  a.mbx = magic(a.bxb);
  a.myc = magic(a.yc);
  a.mrc = magic(a.rc);
  a.cp_pairs = (p.dims[0] % 2 == 0) && (a.bxb % 2 == 0) && (((uintptr_t)d_in & 7) == 0);
  a.jfloor = 5e-2;
  // The tensor map reads the field itself when its x lines are whole
  // multiples of 16 bytes, else the pitched copy the launch writes first (a
  // plan over the whole field); the per-element reads (exact evaluations, raw
  // records, escapes) stay on the field itself.
  const void* tsrc = d_in;
  int64_t pitch = p.dims[0];
  const bool pitched = w.pitched && w.pitch > 0 && blo == 0 && bhi == p.nb && pitched_row(p, true) == w.pitch;
  if (pitched) {
    const int64_t rows = p.nvars * p.dims[3] * p.dims[2] * p.dims[1];
    const int pairs = (p.dims[0] % 2 == 0) && (((uintptr_t)d_in & 7) == 0);
    int dev0 = 0, sms0 = 152;
    if (cudaGetDevice(&dev0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0) != cudaSuccess)
      return DLS_ERR_CUDA;
    const int64_t cap = (int64_t)sms0 * 8, need = cdiv(rows, 8);
    k_pitch_rows<<<(unsigned)(need < cap ? (need > 0 ? need : 1) : cap), 256, 0, s>>>(
        static_cast<const float*>(d_in), w.pitched, rows, p.dims[0], w.pitch, pairs);
    tsrc = w.pitched;
    pitch = w.pitch;
  }
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  const bool aligned = (pitch % 4 == 0) && (p.block[0] % 4 == 0) && (((uintptr_t)tsrc & 15) == 0);
  a.use_tma = 0;
  if (aligned) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc) {
      const cuuint64_t dims[5] = {(cuuint64_t)p.dims[0], (cuuint64_t)p.dims[1], (cuuint64_t)p.dims[2],
                                  (cuuint64_t)p.dims[3], (cuuint64_t)p.nvars};
      const cuuint64_t plane = (cuuint64_t)(pitch * p.dims[1] * p.dims[2]);     // one time step
      const cuuint64_t strides[4] = {(cuuint64_t)pitch * 4, (cuuint64_t)(pitch * p.dims[1]) * 4, plane * 4,
                                     plane * (cuuint64_t)p.dims[3] * 4};
      const cuuint32_t box[5] = {(cuuint32_t)a.bxb, (cuuint32_t)a.yc, (cuuint32_t)a.zc, (cuuint32_t)a.bt, 1u};
      const cuuint32_t es[5] = {1, 1, 1, 1, 1};
      const CUresult rc = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(tsrc), dims, strides, box,
                              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      a.use_tma = rc == CUDA_SUCCESS ? 1 : 0;
    }
  }
  // tensor-core Gram (3xTF32): 16 x 16 x bz x 16 blocks on a TMA-aligned field;
  // the second map stages chunks as [t / 8][y][x / 4][t % 8][x % 4]
  CUtensorMap tmapg;
  memset(&tmapg, 0, sizeof(tmapg));
  a.tc_gram = 0;
  const int tc_mode = p.precision == DLS_PREC_TF32X3 ? kTcTf32x3
                      : p.precision == DLS_PREC_TF32  ? kTcTf32
                      : p.precision == DLS_PREC_BF16X3 ? kTcBf16x3
                      : p.precision == DLS_PREC_BF16  ? kTcBf16
                                                      : kTcNone;
  if (tc_mode != kTcNone && a.use_tma && !pitched && a.bxb == 16 && a.yc == 16 && a.zc == 1 && a.bt == 16) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const cuuint64_t dims[5] = {4, (cuuint64_t)(p.dims[3] * p.nvars), (cuuint64_t)(p.dims[0] / 4), (cuuint64_t)p.dims[1],
                                (cuuint64_t)p.dims[2]};
    const cuuint64_t strides[4] = {(cuuint64_t)p.P * 4, 16, (cuuint64_t)p.dims[0] * 4,
                                   (cuuint64_t)(p.dims[0] * p.dims[1]) * 4};
    const cuuint32_t box[5] = {4, 8, 4, 16, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    if (enc && enc(&tmapg, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(d_in), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      a.tc_gram = tc_mode;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DLS_ERR_CUDA;
  const int64_t nblk = bhi - blo;
  auto grid_of = [&](int per_sm, int cap) -> int {
    int64_t c = (int64_t)sms * per_sm;
    if (cap > 0 && c > cap) c = cap;
    if (c > nblk) c = nblk;
    return (int)(c > 0 ? c : 1);
  };
  const bool tc = a.tc_gram != 0;
  // counters and list of this launch
  if (cudaMemsetAsync(a.ctl, 0, sizeof(FastCtl), s) != cudaSuccess) return DLS_ERR_CUDA;
  // 1. Gram pass (4 CTAs per SM: the staging ring and, with the tensor-core
  //    Gram, the TMEM columns)
  {
    const size_t sm = tile_smem_bytes(tc);
    const int per = tc ? ctas_per_sm_of(k_gram<4, true>, sm, true) : ctas_per_sm_of(k_gram<4, false>, sm, false);
    cudaGetLastError();
    if (per < 1) return DLS_ERR_CUDA;
    const int grid = grid_of(per, w.ctas);
    if (tc) k_gram<4, true><<<grid, kTT, sm, s>>>(tmap, tmapg, a);
    else k_gram<4, false><<<grid, kTT, sm, s>>>(tmap, tmapg, a);
    if (!mark(0)) return DLS_ERR_CUDA;
  }
  // 2. eigensolve and prediction (no staging ring: more CTAs per SM)
  {
    const size_t sm = eig_smem_bytes();
    const int per = ctas_per_sm_of(k_eig<false>, sm, false);
    cudaGetLastError();
    if (per < 1) return DLS_ERR_CUDA;
    k_eig<false><<<grid_of(per, 0), kTT, sm, s>>>(a);
    if (!mark(1)) return DLS_ERR_CUDA;
  }
  // 2b. the Rayleigh-Ritz pass of the flagged blocks: projected Gram, second solve
  {
    const size_t tsm0 = tile_smem_bytes(false);
    const int per = ctas_per_sm_of(k_rrgram<4>, tsm0, false);
    const size_t sm = eig_smem_bytes();
    const int pere = ctas_per_sm_of(k_eig<true>, sm, false);
    cudaGetLastError();
    if (per < 1 || pere < 1) return DLS_ERR_CUDA;
    k_rrgram<4><<<grid_of(per, w.ctas), kTT, tsm0, s>>>(tmap, tmapg, a);
    k_eig<true><<<grid_of(pere, 0), kTT, sm, s>>>(a);
    if (!mark(2)) return DLS_ERR_CUDA;
  }
  // 3. encode pass and deferred record at the predicted rank
  const size_t tsm = tile_smem_bytes(false);
  if (learned != kRankSearch) {
    const int per = occ.whole == 1 ? ctas_per_sm_of(k_enc<2>, tsm, false) : ctas_per_sm_of(k_enc<4>, tsm, false);
    cudaGetLastError();
    if (per < 1) return DLS_ERR_CUDA;
    const int grid = grid_of(per, w.ctas);
    if (occ.whole == 1) k_enc<2><<<grid, kTT, tsm, s>>>(tmap, tmapg, a);
    else k_enc<4><<<grid, kTT, tsm, s>>>(tmap, tmapg, a);
    a.from_list = 1;
  }
  if (!mark(3)) return DLS_ERR_CUDA;
  // 4. the other blocks (all of them with the bisection).  By default the few
  //    k_enc leaves take the 2-CTA form (no spills: 0.334 -> 0.285 ms for the
  //    one block left at 1e-3) and a full search the 4-CTA form; a plan's
  //    tuning picks the form for its own list.
  {
    const int rv = occ.rest != 0 ? occ.rest : (a.from_list ? 1 : 2);
    const int per = tile_ctas_per_sm(rv);
    if (per < 1) return DLS_ERR_CUDA;
    int ctas = sms * per;
    if (ctas > w.ctas) ctas = w.ctas;
    if ((int64_t)ctas > nblk) ctas = (int)nblk;
    if (rv == 1) k_tile<2><<<ctas, kTT, tsm, s>>>(tmap, tmapg, a);
    else k_tile<4><<<ctas, kTT, tsm, s>>>(tmap, tmapg, a);
  }
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

// The deferred records of a compression (after the scan has placed them).
int launch_pack_tile(const Plan& p, const MixedWork& w, const void* d_in, void* d_out, cudaStream_t s) {
  if (p.nb == 0) return DLS_OK;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DLS_ERR_CUDA;
  const int64_t cap = (int64_t)sms * 6;
  const int grid = (int)(p.nb < cap ? p.nb : cap);
  k_pack_tile<<<grid, kTT, 0, s>>>(p, w.meta, w.staging, w.offsets, w.status, (uint8_t*)d_out,
                                   static_cast<const float*>(d_in));
  return cudaGetLastError() == cudaSuccess ? DLS_OK : DLS_ERR_CUDA;
}

}  // namespace dls
