// Host side of the C ABI: parameter validation, block plan, workspace layout,
// launch sequence and status readback.  See include/dls.h for the contract.
#include <atomic>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "dls_internal.cuh"

namespace dls {

static int esize(int dtype) { return dtype == DLS_F32 ? 4 : 8; }

// Same rules as the stream decoder applies to headers.
int make_plan(const dls_params* p, Plan* out) {
  if (!p || p->nvars < 1 || p->nvars > kMaxVars || !p->eb) return DLS_ERR_INVALID_ARG;
  if (p->dtype != DLS_F32 && p->dtype != DLS_F64) return DLS_ERR_INVALID_ARG;
  if (p->eb_type < 0 || p->eb_type > 2 || p->rank_cap < 0) return DLS_ERR_INVALID_ARG;
  if (p->precision < 0 || p->precision > 5 || p->rank_mode < 0 || p->rank_mode > 2) return DLS_ERR_INVALID_ARG;
  if (p->corr_codec != 0 && p->corr_codec != 1) return DLS_ERR_INVALID_ARG;
  for (int a = 0; a < 4; ++a)
    if (p->dims[a] < 1 || p->block[a] < 1 || p->block[a] > p->dims[a]) return DLS_ERR_INVALID_ARG;
  const int64_t M = (int64_t)p->block[0] * p->block[1] * p->block[2];
  const int64_t T = p->block[3];
  if ((M < T ? M : T) > kMaxN) return DLS_ERR_INVALID_ARG;
  if (M * T > (1ll << 26)) return DLS_ERR_INVALID_ARG;
  for (int v = 0; v < p->nvars; ++v)
    if (!(p->eb[v] > 0.0) || !isfinite(p->eb[v])) return DLS_ERR_INVALID_ARG;
  if (p->basis) {
    // a fixed basis (Sec. 4): the plain form with the bisection only, order
    // 1..32, finite entries, columns orthonormal to 1e-12
    if (p->precision != DLS_PREC_FP64 || p->rank_mode != DLS_RANK_SEARCH) return DLS_ERR_INVALID_ARG;
    const int bn = p->basis_n;
    if (bn < 1 || bn > kMaxN) return DLS_ERR_INVALID_ARG;
    for (int i = 0; i < bn; ++i) {
      for (int j = i; j < bn; ++j) {
        double d = 0.0;
        for (int a = 0; a < bn; ++a) {
          if (!isfinite(p->basis[a * bn + i])) return DLS_ERR_INVALID_ARG;
          d = fma(p->basis[a * bn + i], p->basis[a * bn + j], d);
        }
        if (fabs(d - (i == j ? 1.0 : 0.0)) > 1e-12) return DLS_ERR_INVALID_ARG;
      }
    }
  }
  if (p->global_stats) {
    // statistics of the whole field, for a call on one part of it
    const double pts = p->global_stats[3];
    for (int v = 0; v < p->nvars; ++v) {
      const double* g = p->global_stats + 4 * v;
      for (int i = 0; i < 4; ++i)
        if (!isfinite(g[i])) return DLS_ERR_INVALID_ARG;
      if (!(g[0] <= g[1]) || !(g[2] >= 0.0) || !(g[3] >= 1.0) || g[3] != pts || g[3] != floor(g[3]))
        return DLS_ERR_INVALID_ARG;
    }
  }
  Plan P;
  memset(&P, 0, sizeof(P));
  P.basis_n = p->basis ? p->basis_n : 0;
  P.nvars = p->nvars;
  P.dtype = p->dtype;
  P.eb_type = p->eb_type;
  P.rank_cap = p->rank_cap;
  P.precision = p->precision;
  P.rank_mode = p->rank_mode;
  P.nb_total = p->nvars;
  for (int a = 0; a < 4; ++a) {
    P.dims[a] = p->dims[a];
    P.block[a] = p->block[a];
    P.nbk[a] = cdiv(p->dims[a], p->block[a]);
    P.nb_total *= P.nbk[a];
  }
  const int64_t e = p->block_end < 0 ? P.nb_total : p->block_end;
  if (p->block_begin < 0 || p->block_begin > e || e > P.nb_total) return DLS_ERR_INVALID_ARG;
  P.b0 = p->block_begin;
  P.nb = e - p->block_begin;
  P.P = p->dims[0] * p->dims[1] * p->dims[2];
  P.K = P.P * p->dims[3];
  P.has_gstats = p->global_stats ? 1 : 0;
  P.corr_codec = p->corr_codec;
  P.kbound = p->global_stats ? p->global_stats[3] : (double)P.K;
  P.nmax = (int32_t)(M < T ? M : T);
  P.lmax = (int32_t)(M < T ? T : M);
  P.nmax_full = P.nmax;
  P.offsets_pos = align_up(kHdr + (int64_t)kVarRec * p->nvars, 16);
  P.payload_pos = align_up(P.offsets_pos + 8 * (P.nb + 1), 16);
  for (int v = 0; v < p->nvars; ++v) P.eb_user[v] = p->eb[v];
  if (P.nb > 0) {
    const Geom g0 = block_geom(P, P.b0);
    const Geom g1 = block_geom(P, P.b0 + P.nb - 1);
    P.pt_base = g0.pt_off;
    P.pt_count = g1.pt_off + g1.N - g0.pt_off;
  }
  *out = P;
  return DLS_OK;
}

struct Layout {
  size_t meta, vst, q, kc, offsets, vars, status, partial, basis, total;
  // mixed-precision form
  size_t staging, q_scr, k8_scr, k32_scr, bit_scr, feat, ranks, phase, fast;
  size_t gstats;        // nvars x 4 doubles when the caller gives the whole field's statistics
  size_t rice_tmp, rice_info, rice_chunks;   // Rice stage: the packers' stream (bound bytes), per-block
                                             // choices, per-chunk run counts
  size_t pitched;       // the field with padded x lines (MixedWork::pitched)
  int64_t pitch;
  int ctas;
  bool mixed;
};

// The mixed-precision form serves float32 fields with Gram order <= 16.
static bool use_mixed(const Plan& P) {
  return P.precision != DLS_PREC_FP64 && P.dtype == DLS_F32 && P.nmax <= kMaxMixedN;
}

static int mixed_ctas() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  cudaGetLastError();
  return 4 * sms;
}

// Kernels serving the mixed form: k_tile takes the blocks whose Gram side is
// time when its chunk box fits the plan; k_mixed takes the others (or all).
struct MixedRoute {
  bool tile, legacy, spatial_only;
};
static MixedRoute mixed_route(const Plan& P) {
  bool has0 = false, has1 = false;
  for (int c = 0; c < 16; ++c) {
    int64_t s[4];
    bool exists = true;
    for (int a = 0; a < 4; ++a) {
      const int64_t edge = P.dims[a] % P.block[a];
      if (c >> a & 1) {
        if (edge == 0) exists = false;
        s[a] = edge;
      } else {
        if (P.dims[a] < P.block[a]) exists = false;
        s[a] = P.block[a];
      }
    }
    if (!exists) continue;
    const int64_t M = s[0] * s[1] * s[2], T = s[3];
    if (T <= M) has0 = true;
    else has1 = true;
  }
  int bxb, yc, zc, bt;
  const bool fits = tile_chunk_box(P, &bxb, &yc, &zc, &bt);
  MixedRoute r;
  r.tile = fits && has0;
  r.legacy = !fits || has1;
  r.spatial_only = fits;
  return r;
}

static int launch_mixed_all(const Plan& P, const void* d_in, const MixedWork& mw, int mode, Occupancy occ,
                            cudaStream_t s, const cudaEvent_t* pev = nullptr) {
  const MixedRoute rt = mixed_route(P);
  int st;
  if (rt.tile && (st = launch_tile_compress(P, d_in, mw, mode, occ, s, 0, -1, pev)) != DLS_OK) return st;
  if (rt.legacy &&
      (st = launch_mixed_compress(P, d_in, mw, mode, occ.rest != 0 ? occ.rest : 2, rt.spatial_only ? 1 : 0, s)) !=
          DLS_OK)
    return st;
  return DLS_OK;
}

static int64_t bound_bytes(const Plan& P);

static Layout work_layout(const Plan& P) {
  Layout L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (size_t)align_up((int64_t)(off + bytes), 256);
    return o;
  };
  auto take_rice = [&](Layout& l) {
    if (!P.corr_codec) return;
    l.rice_tmp = take((size_t)bound_bytes(P));
    l.rice_info = take(sizeof(RiceInfo) * (size_t)(P.nb > 0 ? P.nb : 1));
    l.rice_chunks = take(sizeof(RiceChunk) * (size_t)(P.nb > 0 ? P.nb : 1) * (size_t)rice_chunks_per_block(P));
  };
  if (use_mixed(P)) {
    const int64_t nb1 = P.nb > 0 ? P.nb : 1;
    const int64_t npt = align_up((int64_t)P.nmax * P.lmax, 16);   // 16-byte rows of k8
    L.mixed = true;
    L.ctas = mixed_ctas();
    L.meta = take(sizeof(BlockMeta) * (size_t)nb1);
    L.offsets = take(sizeof(unsigned long long) * (size_t)(P.nb + 1));
    L.vars = take(sizeof(VarInfo) * kMaxVars);
    L.status = take(sizeof(Status));
    L.partial = take(sizeof(double) * (size_t)stats_partial_doubles(P));
    L.staging = take((size_t)(align_up(P.pt_count * 4, 16) + 48 * nb1 + 64));
    L.q_scr = take(sizeof(int32_t) * (size_t)L.ctas * kMaxMixedN * (size_t)align_up(P.lmax, 4));
    L.k8_scr = take((size_t)L.ctas * (size_t)npt);
    L.k32_scr = take(sizeof(int32_t) * (size_t)L.ctas * (size_t)npt);
    L.bit_scr = take(sizeof(uint32_t) * (size_t)L.ctas * (size_t)(align_up(npt, 32) / 32));
    L.feat = take(sizeof(float) * 32 * (size_t)nb1);
    L.ranks = take(sizeof(int32_t) * (size_t)nb1);
    L.phase = take(sizeof(unsigned long long) * (size_t)L.ctas * kMixedPhases);
    L.fast = take(tile_fast_bytes(P.nb));
    L.gstats = P.has_gstats ? take(sizeof(double) * 4 * (size_t)P.nvars) : 0;
    L.pitch = pitched_row(P, mixed_route(P).tile);
    L.pitched = L.pitch ? take(sizeof(float) * (size_t)(P.nvars * P.dims[3] * P.dims[2] * P.dims[1] * L.pitch)) : 0;
    take_rice(L);
    L.total = off;
    return L;
  }
  L.meta = take(sizeof(BlockMeta) * (size_t)(P.nb > 0 ? P.nb : 1));
  L.vst = take(sizeof(double) * (size_t)(P.nb > 0 ? P.nb : 1) * P.nmax * P.nmax);
  L.q = take(sizeof(int32_t) * (size_t)(P.pt_count > 0 ? P.pt_count : 1));
  L.kc = take(sizeof(int32_t) * (size_t)(P.pt_count > 0 ? P.pt_count : 1));
  L.offsets = take(sizeof(unsigned long long) * (size_t)(P.nb + 1));
  L.vars = take(sizeof(VarInfo) * kMaxVars);
  L.status = take(sizeof(Status));
  L.partial = take(sizeof(double) * (size_t)stats_partial_doubles(P));
  L.basis = P.basis_n > 0 ? take(sizeof(double) * (size_t)P.basis_n * P.basis_n) : 0;
  L.gstats = P.has_gstats ? take(sizeof(double) * 4 * (size_t)P.nvars) : 0;
  take_rice(L);
  L.total = off;
  return L;
}

static Work carve(const Layout& L, void* ws) {
  uint8_t* b = (uint8_t*)ws;
  Work w;
  w.meta = (BlockMeta*)(b + L.meta);
  w.vst = (double*)(b + L.vst);
  w.q = (int32_t*)(b + L.q);
  w.kc = (int32_t*)(b + L.kc);
  w.offsets = (unsigned long long*)(b + L.offsets);
  w.vars = (VarInfo*)(b + L.vars);
  w.status = (Status*)(b + L.status);
  w.basis = L.basis ? (const double*)(b + L.basis) : nullptr;
  w.gstats = L.gstats ? (const double*)(b + L.gstats) : nullptr;
  return w;
}

// Copies the fixed basis (if any) into its workspace region, stream-ordered;
// the host array may be freed once this returns.
static int upload_basis(const dls_params* p, const Plan& P, const Layout& L, void* d_ws, cudaStream_t s) {
  if (P.has_gstats) {
    // the whole field's statistics (small; copied with the basis, before any kernel reads them)
    if (cudaMemcpyAsync((uint8_t*)d_ws + L.gstats, p->global_stats, sizeof(double) * 4 * (size_t)P.nvars,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return DLS_ERR_CUDA;
  }
  if (P.basis_n == 0) return DLS_OK;
  const size_t bytes = sizeof(double) * (size_t)P.basis_n * P.basis_n;
  return cudaMemcpyAsync((uint8_t*)d_ws + L.basis, p->basis, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess
             ? DLS_OK
             : DLS_ERR_CUDA;
}

static int64_t bound_bytes(const Plan& P) {
  int64_t tot = P.payload_pos;
  const int es = esize(P.dtype);
  // records of blocks sharing a shape have equal bounds: sum per block
  for (int64_t b = 0; b < P.nb; ++b) tot += raw_record_bytes(block_geom(P, P.b0 + b).N, es);
  return tot;
}

#define CK(x)                                  \
  do {                                         \
    if ((x) != cudaSuccess) return DLS_ERR_CUDA; \
  } while (0)

struct HostHeader {
  dls_params p;
  double eb_user[kMaxVars], eb[kMaxVars], delta[kMaxVars], step[kMaxVars];
  int64_t offsets_pos, payload_pos, total, total_blocks;
  int32_t precision, rank_mode, version;
};

// Reads and validates a stream header from device memory.
static int read_header(const void* d_comp, size_t comp_bytes, cudaStream_t s, HostHeader* h, Plan* P) {
  if (!d_comp || comp_bytes < (size_t)kHdr || ((uintptr_t)d_comp & 15)) return DLS_ERR_INVALID_ARG;
  uint8_t hdr[kHdr];
  CK(cudaMemcpyAsync(hdr, d_comp, kHdr, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  uint32_t u32[32];
  uint64_t u64[16];
  memcpy(u32, hdr, kHdr);
  memcpy(u64, hdr, kHdr);
  if (u32[0] != kMagic || u32[1] != kVersion || u32[2] != (uint32_t)kHdr) return DLS_ERR_CORRUPT;
  const int nvars = (int)u32[3];
  if (nvars < 1 || nvars > kMaxVars) return DLS_ERR_CORRUPT;
  if ((size_t)(kHdr + kVarRec * nvars) > comp_bytes) return DLS_ERR_CORRUPT;
  std::vector<double> vt(4 * (size_t)nvars);
  CK(cudaMemcpyAsync(vt.data(), (const uint8_t*)d_comp + kHdr, kVarRec * (size_t)nvars, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  memset(h, 0, sizeof(*h));
  for (int v = 0; v < nvars; ++v) {
    h->eb_user[v] = vt[4 * v + 0];
    h->eb[v] = vt[4 * v + 1];
    h->delta[v] = vt[4 * v + 2];
    h->step[v] = vt[4 * v + 3];
  }
  dls_params& p = h->p;
  p.nvars = nvars;
  for (int a = 0; a < 4; ++a) p.dims[a] = (int64_t)u64[2 + a];
  for (int a = 0; a < 4; ++a) p.block[a] = (int32_t)u32[12 + a];
  p.dtype = hdr[64];
  p.eb_type = hdr[65];
  h->precision = hdr[66];
  h->rank_mode = hdr[67];
  h->version = (int32_t)u32[1];
  p.precision = 0;
  p.rank_mode = 0;
  p.rank_cap = (int32_t)u32[17];
  p.block_begin = (int64_t)u64[9];
  p.block_end = (int64_t)u64[10];
  p.eb = h->eb_user;
  p.basis = nullptr;   // records carry their modes
  p.basis_n = 0;
  h->total_blocks = (int64_t)u64[11];
  h->offsets_pos = (int64_t)u64[13];
  h->payload_pos = (int64_t)u64[14];
  h->total = (int64_t)u64[15];
  if (make_plan(&p, P) != DLS_OK) return DLS_ERR_CORRUPT;
  if (h->total_blocks != P->nb_total || (int64_t)u64[12] != kHdr || h->offsets_pos != P->offsets_pos ||
      h->payload_pos != P->payload_pos || h->total != (int64_t)comp_bytes || h->payload_pos > h->total)
    return DLS_ERR_CORRUPT;
  for (int v = 0; v < nvars; ++v) {
    const bool pointwise = p.eb_type != DLS_EB_NRMSE;
    if (!(h->delta[v] > 0.0) || !isfinite(h->delta[v]) || !isfinite(h->step[v]) ||
        (pointwise && !(h->eb[v] > 0.0)))
      return DLS_ERR_CORRUPT;
  }
  return DLS_OK;
}

static MixedWork mixed_work(const Plan& P, const Layout& L, void* ws) {
  uint8_t* b = (uint8_t*)ws;
  const Work w = carve(L, ws);
  MixedWork mw;
  mw.meta = w.meta;
  mw.offsets = w.offsets;
  mw.vars = w.vars;
  mw.status = w.status;
  mw.staging = b + L.staging;
  mw.q_scr = (int32_t*)(b + L.q_scr);
  mw.k8_scr = (int8_t*)(b + L.k8_scr);
  mw.k32_scr = (int32_t*)(b + L.k32_scr);
  mw.bit_scr = (uint32_t*)(b + L.bit_scr);
  mw.feat = (float*)(b + L.feat);
  mw.ranks = (int32_t*)(b + L.ranks);
  mw.lmax = align_up(P.lmax, 4);
  mw.nptmax = align_up((int64_t)P.nmax * P.lmax, 16);
  mw.ctas = L.ctas;
  mw.phase = (unsigned long long*)(b + L.phase);
  mw.fast = b + L.fast;
  mw.pitched = L.pitch ? (float*)(b + L.pitched) : nullptr;
  mw.pitch = L.pitch;
  return mw;
}

// Enqueues the whole compression on `s` (no host synchronisation): status
// reset, bound resolution, the per-block kernel of the chosen form, the scan
// writing header and offset table, and the record packer / compaction.
// ev0 / ev1 (optional) bracket the per-block kernels; pev (optional, five
// events) marks the ends of k_gram, k_eig, the Rayleigh-Ritz kernels, k_enc
// and of the record packing.
static int enqueue_compress(const Plan& P, const Layout& L, const void* d_in, void* d_out, size_t out_cap,
                            void* d_ws, Occupancy occ, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                            cudaEvent_t ev1 = nullptr, const cudaEvent_t* pev = nullptr) {
  int st;
  Work w = carve(L, d_ws);
  CK(cudaMemsetAsync(w.status, 0, sizeof(Status), s));
  // with the Rice stage the packers write into its staging stream, which the
  // stage then rewrites into d_out
  void* out1 = P.corr_codec ? (void*)((uint8_t*)d_ws + L.rice_tmp) : d_out;
  const size_t cap1 = P.corr_codec ? (size_t)bound_bytes(P) : out_cap;
  double* partial = (double*)((uint8_t*)d_ws + L.partial);
  if ((st = launch_stats_resolve(P, d_in, w, partial, s)) != DLS_OK) return st;
  if (L.mixed) {
    const MixedWork mw = mixed_work(P, L, d_ws);
    CK(cudaMemsetAsync(mw.phase, 0, sizeof(unsigned long long) * (size_t)L.ctas * kMixedPhases, s));
    const int mode = P.rank_mode == DLS_RANK_LEARNED ? kRankMlp : (P.rank_mode == DLS_RANK_TAIL ? kRankTail : kRankSearch);
    if (ev0) CK(record_marker(ev0, s));
    if ((st = launch_mixed_all(P, d_in, mw, mode, occ, s, pev)) != DLS_OK) return st;
    if (ev1) CK(record_marker(ev1, s));
    if ((st = launch_scan(P, w, cap1, out1, s)) != DLS_OK) return st;
    if ((st = launch_compact(P, mw, out1, s)) != DLS_OK) return st;
    if ((st = launch_pack_tile(P, mw, d_in, out1, s)) != DLS_OK) return st;
  } else {
    if (ev0) CK(record_marker(ev0, s));
    if ((st = launch_plain_compress(P, d_in, w, s)) != DLS_OK) return st;
    if (ev1) CK(record_marker(ev1, s));
    if ((st = launch_scan(P, w, cap1, out1, s)) != DLS_OK) return st;
    if ((st = launch_pack(P, d_in, w, out1, cap1, s)) != DLS_OK) return st;
  }
  if (P.corr_codec &&
      (st = launch_rice(P, w, (const uint8_t*)out1, (RiceInfo*)((uint8_t*)d_ws + L.rice_info),
                        (RiceChunk*)((uint8_t*)d_ws + L.rice_chunks), out_cap, d_out, s)) != DLS_OK)
    return st;
  if (L.mixed && pev && pev[4]) CK(record_marker(pev[4], s));
  return DLS_OK;
}

// Host-buffer compression with the copy of each slab of the field overlapped
// with the compression of the slabs before it.  Blocks are ordered (variable,
// time block, z, y, x) and the field (variable, t, z, y, x), so the blocks of
// one slab of block[3] time steps of one variable are a contiguous range and
// their values a contiguous byte range.  Taken for the mixed forms with an
// absolute bound (no pass over the whole field first) whose blocks all go
// through the tile kernel, over the whole block range.
static bool host_pipelined(const Plan& P, const Layout& L) {
  return L.mixed && P.eb_type == DLS_EB_ABS && !mixed_route(P).legacy && P.b0 == 0 && P.nb == P.nb_total &&
         P.nvars * P.nbk[3] >= 2;
}
static int compress_host_pipelined(const Plan& P, const Layout& L, const void* h_in, uint8_t* d_in,
                                   uint8_t* d_out, size_t bound, uint8_t* d_ws, cudaStream_t s, size_t* nb_out) {
  int st;
  Work w = carve(L, d_ws);
  const MixedWork mw = mixed_work(P, L, d_ws);
  const int mode = P.rank_mode == DLS_RANK_LEARNED ? kRankMlp : (P.rank_mode == DLS_RANK_TAIL ? kRankTail : kRankSearch);
  const int64_t nseg = (int64_t)P.nvars * P.nbk[3];
  const int64_t nbs = P.nbk[0] * P.nbk[1] * P.nbk[2];      // blocks of one slab
  const size_t es = (size_t)esize(P.dtype);
  cudaStream_t cs = nullptr;
  cudaEvent_t* ev = new cudaEvent_t[nseg]();
  auto done = [&](int rc) {
    for (int64_t k = 0; k < nseg; ++k)
      if (ev[k]) cudaEventDestroy(ev[k]);
    delete[] ev;
    if (cs) cudaStreamDestroy(cs);
    return rc;
  };
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return done(DLS_ERR_CUDA);
  for (int64_t k = 0; k < nseg; ++k)
    if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) return done(DLS_ERR_CUDA);
  // the copies, slab by slab, on their own stream
  for (int64_t k = 0; k < nseg; ++k) {
    const int64_t v = k / P.nbk[3], tb = k % P.nbk[3];
    const int64_t t0 = tb * P.block[3], t1 = (t0 + P.block[3]) < P.dims[3] ? t0 + P.block[3] : P.dims[3];
    const size_t off = (size_t)(v * P.K + t0 * P.P) * es, len = (size_t)((t1 - t0) * P.P) * es;
    if (cudaMemcpyAsync(d_in + off, (const uint8_t*)h_in + off, len, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(ev[k], cs) != cudaSuccess)
      return done(DLS_ERR_CUDA);
  }
  // the compression: each slab's blocks once its copy has landed
  if (cudaMemsetAsync(w.status, 0, sizeof(Status), s) != cudaSuccess) return done(DLS_ERR_CUDA);
  if ((st = launch_stats_resolve(P, d_in, w, (double*)(d_ws + L.partial), s)) != DLS_OK) return done(st);
  if (cudaMemsetAsync(mw.phase, 0, sizeof(unsigned long long) * (size_t)L.ctas * kMixedPhases, s) != cudaSuccess)
    return done(DLS_ERR_CUDA);
  for (int64_t k = 0; k < nseg; ++k) {
    if (cudaStreamWaitEvent(s, ev[k], 0) != cudaSuccess ||
        cudaMemsetAsync(&w.status->pad[1], 0, sizeof(unsigned long long), s) != cudaSuccess)
      return done(DLS_ERR_CUDA);
    if ((st = launch_tile_compress(P, d_in, mw, mode, kOccDefault, s, k * nbs, (k + 1) * nbs)) != DLS_OK) return done(st);
  }
  uint8_t* out1 = P.corr_codec ? d_ws + L.rice_tmp : d_out;
  if ((st = launch_scan(P, w, bound, out1, s)) != DLS_OK) return done(st);
  if ((st = launch_compact(P, mw, out1, s)) != DLS_OK) return done(st);
  if ((st = launch_pack_tile(P, mw, d_in, out1, s)) != DLS_OK) return done(st);
  if (P.corr_codec && (st = launch_rice(P, w, out1, (RiceInfo*)(d_ws + L.rice_info),
                                        (RiceChunk*)(d_ws + L.rice_chunks), bound, d_out, s)) != DLS_OK)
    return done(st);
  Status hs;
  if (cudaMemcpyAsync(&hs, w.status, sizeof(Status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(DLS_ERR_CUDA);
  if (hs.timeout) return done(DLS_ERR_TIMEOUT);
  if (hs.nonfinite) return done(DLS_ERR_NONFINITE);
  *nb_out = (size_t)hs.total_bytes;
  if (hs.capacity) return done(DLS_ERR_CAPACITY);
  return done(hs.corrupt ? DLS_ERR_CORRUPT : DLS_OK);
}

}  // namespace dls

// ---------------------------------------------------------------- plans: autotune + CUDA graph
struct dls_plan {
  dls::Plan P;
  dls::Layout L;
  const void* d_in;
  void* d_out;
  size_t out_cap;
  void* d_ws;
  dls::Occupancy occ;
  float tune_ms[3];        // [1], [2]: a whole compression with every class in form 1, in form 2
  float class_ms[2][2];    // [class][form - 1]: device ms of the class's kernels (whole, rest)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  dls::Status* h_status;   // pinned
  cudaEvent_t kev[2];      // recorded around the per-block kernels inside the graph
  cudaEvent_t pev[5];      // ends of k_gram, k_eig, the Rayleigh-Ritz kernels, k_enc, the record packing
  int kernel_nodes;
};

namespace dls {

static std::string tune_key(const Plan& P) {
  int dev = 0;
  cudaDeviceProp prop;
  memset(&prop, 0, sizeof(prop));
  if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|nv%d|d%lldx%lldx%lldx%lld|b%dx%dx%dx%d|t%d|e%d|p%d|r%d|c%d", prop.name,
           prop.multiProcessorCount, P.nvars, (long long)P.dims[0], (long long)P.dims[1], (long long)P.dims[2],
           (long long)P.dims[3], P.block[0], P.block[1], P.block[2], P.block[3], P.dtype, P.eb_type, P.precision,
           P.rank_mode, P.rank_cap);
  for (char* c = buf; *c; ++c)
    if (*c == '"' || *c == '\\') *c = '_';
  return std::string(buf);
}

static const char* tune_cache_path() {
  const char* e = getenv("DLS_AUTOTUNE_CACHE");
  return (e && *e) ? e : nullptr;
}

// Cached form for the key (JSON lines {"key": "...", "variant": v, ...}; the
// last line for a key wins), or 0.  A plan's keys are its parameters' key
// followed by "|whole" and "|rest", one line per shape class.
static int tune_lookup(const std::string& key) {
  const char* path = tune_cache_path();
  if (!path) return 0;
  FILE* f = fopen(path, "r");
  if (!f) return 0;
  char line[2048];
  int found = 0;
  const std::string pat = "\"key\": \"" + key + "\"";
  while (fgets(line, sizeof(line), f)) {
    if (strstr(line, pat.c_str())) {
      const char* v = strstr(line, "\"variant\": ");
      if (v) found = atoi(v + 11);
    }
  }
  fclose(f);
  return (found == 1 || found == 2) ? found : 0;
}

static void tune_store(const std::string& key, int variant, const float* ms) {
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"ms\": [%.4f, %.4f]}\n", key.c_str(), variant, ms[0], ms[1]);
  fclose(f);
}

}  // namespace dls

namespace dls {
namespace {
std::atomic<int64_t> g_withheld{-1};
}
int64_t fault_withheld_block() { return g_withheld.load(); }
}  // namespace dls

using namespace dls;

extern "C" {

const char* dls_status_string(int st) {
  switch (st) {
    case DLS_OK: return "ok";
    case DLS_ERR_INVALID_ARG: return "invalid argument";
    case DLS_ERR_CAPACITY: return "output buffer too small";
    case DLS_ERR_NONFINITE: return "non-finite value in input";
    case DLS_ERR_CORRUPT: return "corrupt stream";
    case DLS_ERR_CUDA: return "CUDA runtime error";
    case DLS_ERR_TIMEOUT: return "device wait timed out";
    case DLS_ERR_BOUND_VIOLATED: return "error bound violated";
    case DLS_ERR_WORKSPACE: return "workspace missing or too small";
    case DLS_ERR_NO_MODEL: return "no rank model loaded";
    default: return "unknown status";
  }
}

size_t dls_compress_bound(const dls_params* p) {
  Plan P;
  if (make_plan(p, &P) != DLS_OK) return 0;
  return (size_t)bound_bytes(P);
}

size_t dls_workspace_size(const dls_params* p) {
  Plan P;
  if (make_plan(p, &P) != DLS_OK) return 0;
  return work_layout(P).total;
}

int dls_compress(const dls_params* p, const void* d_in, void* d_out, size_t out_cap, size_t* out_bytes,
                 void* d_workspace, size_t ws_bytes, dls_stream_t stream) {
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  if (!d_in || !d_out || !out_bytes || ((uintptr_t)d_out & 15) || ((uintptr_t)d_in & (esize(P.dtype) - 1)))
    return DLS_ERR_INVALID_ARG;
  const Layout L = work_layout(P);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  if (L.mixed && P.rank_mode == DLS_RANK_LEARNED && !rank_model_loaded()) return DLS_ERR_NO_MODEL;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(L, d_workspace);
  if ((st = upload_basis(p, P, L, d_workspace, s)) != DLS_OK) return st;
  if ((st = enqueue_compress(P, L, d_in, d_out, out_cap, d_workspace, kOccDefault, s)) != DLS_OK) return st;
  Status hs;
  CK(cudaMemcpyAsync(&hs, w.status, sizeof(Status), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs.timeout) return DLS_ERR_TIMEOUT;
  if (hs.nonfinite) return DLS_ERR_NONFINITE;
  *out_bytes = (size_t)hs.total_bytes;
  if (hs.capacity) return DLS_ERR_CAPACITY;
  return hs.corrupt ? DLS_ERR_CORRUPT : DLS_OK;
}

size_t dls_host_staging_size(const dls_params* p) {
  Plan P;
  if (make_plan(p, &P) != DLS_OK) return 0;
  const size_t in = (size_t)align_up(P.K * P.nvars * esize(P.dtype), 256);
  const size_t out = (size_t)align_up(bound_bytes(P), 256);
  return in + out + work_layout(P).total;
}

int dls_compress_host(const dls_params* p, const void* h_in, void* h_out, size_t out_cap, size_t* out_bytes,
                      void* d_staging, size_t staging_bytes, dls_stream_t stream) {
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  if (!h_in || !h_out || !out_bytes || !d_staging || ((uintptr_t)d_staging & 255)) return DLS_ERR_INVALID_ARG;
  const size_t inb = (size_t)(P.K * P.nvars * esize(P.dtype));
  const size_t in = (size_t)align_up((int64_t)inb, 256);
  const size_t bound = (size_t)bound_bytes(P);
  const size_t out = (size_t)align_up((int64_t)bound, 256);
  const size_t ws = work_layout(P).total;
  if (staging_bytes < in + out + ws) return DLS_ERR_WORKSPACE;
  uint8_t* base = (uint8_t*)d_staging;
  cudaStream_t s = (cudaStream_t)stream;
  size_t nb = 0;
  const Layout L = work_layout(P);
  if (host_pipelined(P, L)) {
    if (L.mixed && P.rank_mode == DLS_RANK_LEARNED && !rank_model_loaded()) return DLS_ERR_NO_MODEL;
    if ((st = upload_basis(p, P, L, base + in + out, s)) != DLS_OK) return st;
    st = compress_host_pipelined(P, L, h_in, base, base + in, bound, base + in + out, s, &nb);
  } else {
    CK(cudaMemcpyAsync(base, h_in, inb, cudaMemcpyHostToDevice, s));
    st = dls_compress(p, base, base + in, bound, &nb, base + in + out, ws, stream);
  }
  *out_bytes = nb;
  if (st != DLS_OK) return st;
  if (nb > out_cap) return DLS_ERR_CAPACITY;
  CK(cudaMemcpyAsync(h_out, base + in, nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return DLS_OK;
}

int dls_decompress(const void* d_comp, size_t comp_bytes, void* d_out, size_t out_cap, dls_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  HostHeader h;
  Plan P;
  int st = read_header(d_comp, comp_bytes, s, &h, &P);
  if (st != DLS_OK) return st;
  if (!d_out || ((uintptr_t)d_out & (esize(P.dtype) - 1))) return DLS_ERR_INVALID_ARG;
  if (out_cap < (size_t)(P.K * P.nvars * esize(P.dtype))) return DLS_ERR_CAPACITY;
  Status* dst = nullptr;
  CK(cudaMallocAsync((void**)&dst, sizeof(Status), s));
  CK(cudaMemsetAsync(dst, 0, sizeof(Status), s));
  st = launch_decode(P, d_comp, (unsigned long long)comp_bytes, d_out, dst, s);
  Status hs;
  memset(&hs, 0, sizeof(hs));
  cudaMemcpyAsync(&hs, dst, sizeof(Status), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(dst, s);
  CK(cudaStreamSynchronize(s));
  if (st != DLS_OK) return st;
  return hs.corrupt ? DLS_ERR_CORRUPT : DLS_OK;
}

int dls_field_stats(const dls_params* p, const void* d_in, double* h_stats, void* d_workspace, size_t ws_bytes,
                    dls_stream_t stream) {
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  if (!d_in || !h_stats || ((uintptr_t)d_in & (esize(P.dtype) - 1))) return DLS_ERR_INVALID_ARG;
  const Layout L = work_layout(P);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(L, d_workspace);
  CK(cudaMemsetAsync(w.status, 0, sizeof(Status), s));
  if ((st = launch_field_stats(P, d_in, w, (double*)((uint8_t*)d_workspace + L.partial), h_stats, s)) != DLS_OK)
    return st;
  Status hs;
  CK(cudaMemcpyAsync(&hs, w.status, sizeof(Status), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return hs.nonfinite ? DLS_ERR_NONFINITE : DLS_OK;
}

int dls_block_features(const dls_params* p, const void* d_in, float* d_feat, int32_t* d_rank, void* d_workspace,
                       size_t ws_bytes, dls_stream_t stream) {
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  if (!d_in || !d_feat || !d_rank || !use_mixed(P)) return DLS_ERR_INVALID_ARG;
  const Layout L = work_layout(P);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(L, d_workspace);
  uint8_t* b = (uint8_t*)d_workspace;
  if ((st = upload_basis(p, P, L, d_workspace, s)) != DLS_OK) return st;
  CK(cudaMemsetAsync(w.status, 0, sizeof(Status), s));
  if ((st = launch_stats_resolve(P, d_in, w, (double*)(b + L.partial), s)) != DLS_OK) return st;
  // the workspace as a compression uses it, with the caller's feature and rank arrays
  MixedWork mw = mixed_work(P, L, d_workspace);
  mw.feat = d_feat;
  mw.ranks = d_rank;
  if ((st = launch_mixed_all(P, d_in, mw, kRankSearch, kOccDefault, s)) != DLS_OK) return st;
  Status hs;
  CK(cudaMemcpyAsync(&hs, w.status, sizeof(Status), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs.timeout) return DLS_ERR_TIMEOUT;
  return hs.nonfinite ? DLS_ERR_NONFINITE : DLS_OK;
}

int dls_mlp_forward(const float* d_params, const float* d_feat, int64_t n, float* d_y, dls_stream_t stream) {
  if (!d_params || n < 0 || (n > 0 && (!d_feat || !d_y))) return DLS_ERR_INVALID_ARG;
  int st = launch_mlp_forward(d_params, d_feat, n, d_y, (cudaStream_t)stream);
  if (st != DLS_OK) return st;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return DLS_OK;
}

int dls_mlp_grad(const float* d_params, const float* d_feat, const float* d_target, int64_t n, float* d_grad,
                 float* d_loss, dls_stream_t stream) {
  if (!d_params || !d_feat || !d_target || !d_grad || !d_loss || n < 1 || n > mlp_max_batch())
    return DLS_ERR_INVALID_ARG;
  int st = launch_mlp_grad(d_params, d_feat, d_target, (int)n, d_grad, d_loss, (cudaStream_t)stream);
  if (st != DLS_OK) return st;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return DLS_OK;
}

int dls_mlp_train(float* d_params, float* d_adam, const float* d_feat, const float* d_target, const int32_t* d_order,
                  int64_t n_order, int32_t steps, int32_t batch, float lr, int32_t step0, float* d_loss,
                  dls_stream_t stream) {
  if (!d_params || !d_adam || !d_feat || !d_target || !d_order || n_order < 1 || steps < 0 || batch < 1 ||
      batch > mlp_max_batch() || !(lr > 0.0f) || step0 < 0)
    return DLS_ERR_INVALID_ARG;
  int st = launch_mlp_train(d_params, d_adam, d_feat, d_target, d_order, n_order, steps, batch, lr, step0, d_loss,
                            (cudaStream_t)stream);
  if (st != DLS_OK) return st;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return DLS_OK;
}

int dls_set_fault_hook(int32_t kind, int64_t arg) {
  if (kind == DLS_FAULT_NONE) {
    g_withheld.store(-1);
    return DLS_OK;
  }
  if (kind != DLS_FAULT_WITHHOLD_CHUNK || arg < 0) return DLS_ERR_INVALID_ARG;
  g_withheld.store(arg);
  return DLS_OK;
}

int dls_stage_quantize(const float* d_c, int64_t n, double delta, int32_t* d_q, int32_t* d_ovf,
                       dls_stream_t stream) {
  if (n < 0 || (n > 0 && (!d_c || !d_q || !d_ovf)) || !(delta > 0.0) || !isfinite(delta)) return DLS_ERR_INVALID_ARG;
  int st = launch_stage_quantize(d_c, n, delta, d_q, d_ovf, (cudaStream_t)stream);
  if (st != DLS_OK) return st;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return DLS_OK;
}

int dls_stage_correct(const float* d_x, const float* d_xh, int64_t n, double eb, int32_t* d_k, dls_stream_t stream) {
  return dls_stage_correct_path(d_x, d_xh, n, eb, DLS_CORR_PATH_EXACT, d_k, stream);
}

int dls_stage_correct_path(const float* d_x, const float* d_xh, int64_t n, double eb, int32_t path, int32_t* d_k,
                           dls_stream_t stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_xh || !d_k)) || !(eb > 0.0) || !isfinite(eb) || path < DLS_CORR_PATH_EXACT ||
      path > DLS_CORR_PATH_DENSE)
    return DLS_ERR_INVALID_ARG;
  int st = launch_stage_correct(d_x, d_xh, n, eb, path, d_k, (cudaStream_t)stream);
  if (st != DLS_OK) return st;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return DLS_OK;
}

int dls_plan_create(const dls_params* p, const void* d_in, void* d_out, size_t out_cap, void* d_workspace,
                    size_t ws_bytes, dls_stream_t stream, dls_plan** out_plan) {
  if (!out_plan) return DLS_ERR_INVALID_ARG;
  *out_plan = nullptr;
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  if (!d_in || !d_out || ((uintptr_t)d_out & 15) || ((uintptr_t)d_in & (esize(P.dtype) - 1)))
    return DLS_ERR_INVALID_ARG;
  const Layout L = work_layout(P);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  if (L.mixed && P.rank_mode == DLS_RANK_LEARNED && !rank_model_loaded()) return DLS_ERR_NO_MODEL;
  cudaStream_t s = (cudaStream_t)stream;
  dls_plan* pl = new dls_plan();
  pl->P = P;
  pl->L = L;
  pl->d_in = d_in;
  pl->d_out = d_out;
  pl->out_cap = out_cap;
  pl->d_ws = d_workspace;
  pl->occ = kOccDefault;
  pl->tune_ms[0] = pl->tune_ms[1] = pl->tune_ms[2] = 0.0f;
  for (int c = 0; c < 2; ++c) pl->class_ms[c][0] = pl->class_ms[c][1] = 0.0f;
  pl->graph = nullptr;
  pl->exec = nullptr;
  pl->h_status = nullptr;
  pl->kev[0] = pl->kev[1] = nullptr;
  for (int i = 0; i < 5; ++i) pl->pev[i] = nullptr;
  pl->kernel_nodes = 0;
  auto fail = [&](int code) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->h_status) cudaFreeHost(pl->h_status);
    for (int i = 0; i < 2; ++i)
      if (pl->kev[i]) cudaEventDestroy(pl->kev[i]);
    for (int i = 0; i < 5; ++i)
      if (pl->pev[i]) cudaEventDestroy(pl->pev[i]);
    delete pl;
    return code;
  };
  if (cudaEventCreate(&pl->kev[0]) != cudaSuccess || cudaEventCreate(&pl->kev[1]) != cudaSuccess)
    return fail(DLS_ERR_CUDA);
  for (int i = 0; i < 5; ++i)
    if (cudaEventCreate(&pl->pev[i]) != cudaSuccess) return fail(DLS_ERR_CUDA);
  if (cudaHostAlloc((void**)&pl->h_status, sizeof(Status), cudaHostAllocDefault) != cudaSuccess) return fail(DLS_ERR_CUDA);
  // the fixed basis goes into the workspace once, outside the captured graph
  if ((st = upload_basis(p, P, L, d_workspace, s)) != DLS_OK) return fail(st);
  if ((P.basis_n > 0 || P.has_gstats) && cudaStreamSynchronize(s) != cudaSuccess) return fail(DLS_ERR_CUDA);
  // autotune, per shape class: run every class in form 1, then every class in
  // form 2 (a warm-up compression, then a timed one), time each class's
  // kernels with the events between the stages, and keep each class's faster
  // form.  The classes run in separate kernels one after the other, and the
  // rest class's list does not depend on the form k_enc ran in, so the two
  // choices are independent.
  if (L.mixed) {
    const std::string key = tune_key(P);
    const std::string kc[2] = {key + "|whole", key + "|rest"};
    int v[2] = {tune_lookup(kc[0]), tune_lookup(kc[1])};
    if (v[0] == 0 || v[1] == 0) {
      const bool staged = mixed_route(P).tile;
      for (int form = 1; form <= 2; ++form) {
        const Occupancy o{form, form};
        if ((st = enqueue_compress(P, L, d_in, d_out, out_cap, d_workspace, o, s)) != DLS_OK) return fail(st);
        if ((st = enqueue_compress(P, L, d_in, d_out, out_cap, d_workspace, o, s, pl->kev[0], pl->kev[1],
                                   pl->pev)) != DLS_OK)
          return fail(st);
        if (cudaEventSynchronize(pl->pev[4]) != cudaSuccess) return fail(DLS_ERR_CUDA);
        float whole = 0.0f, rest = 0.0f;
        if (staged) {
          // k_enc between the Rayleigh-Ritz stage and its own end; k_tile and
          // k_mixed from there to the end of the per-block kernels
          if (cudaEventElapsedTime(&whole, pl->pev[2], pl->pev[3]) != cudaSuccess ||
              cudaEventElapsedTime(&rest, pl->pev[3], pl->kev[1]) != cudaSuccess)
            return fail(DLS_ERR_CUDA);
        } else if (cudaEventElapsedTime(&rest, pl->kev[0], pl->kev[1]) != cudaSuccess) {
          return fail(DLS_ERR_CUDA);
        }
        if (cudaEventElapsedTime(&pl->tune_ms[form], pl->kev[0], pl->pev[4]) != cudaSuccess) return fail(DLS_ERR_CUDA);
        pl->class_ms[0][form - 1] = whole;
        pl->class_ms[1][form - 1] = rest;
      }
      for (int c = 0; c < 2; ++c) {
        v[c] = pl->class_ms[c][0] < pl->class_ms[c][1] ? 1 : 2;
        tune_store(kc[c], v[c], pl->class_ms[c]);
      }
    }
    pl->occ = Occupancy{v[0], v[1]};
  }
  // capture the sequence, ending with the status copy into pinned memory, on a
  // private stream (the legacy default stream cannot be captured)
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(DLS_ERR_CUDA);
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(DLS_ERR_CUDA);
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(DLS_ERR_CUDA);
  }
  st = enqueue_compress(P, L, d_in, d_out, out_cap, d_workspace, pl->occ, cs, pl->kev[0], pl->kev[1],
                        L.mixed ? pl->pev : nullptr);
  Work w = carve(L, d_workspace);
  cudaError_t ce = cudaMemcpyAsync(pl->h_status, w.status, sizeof(Status), cudaMemcpyDeviceToHost, cs);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != DLS_OK || ce != cudaSuccess || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return fail(st != DLS_OK ? st : DLS_ERR_CUDA);
  }
  pl->graph = g;
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++pl->kernel_nodes;
      }
  }
  if (cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) return fail(DLS_ERR_CUDA);
  *out_plan = pl;
  return DLS_OK;
}

int dls_plan_execute(dls_plan* pl, size_t* out_bytes, dls_stream_t stream) {
  if (!pl || !out_bytes) return DLS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaGraphLaunch(pl->exec, s));
  CK(cudaStreamSynchronize(s));
  const Status hs = *pl->h_status;
  if (hs.timeout) return DLS_ERR_TIMEOUT;
  if (hs.nonfinite) return DLS_ERR_NONFINITE;
  *out_bytes = (size_t)hs.total_bytes;
  if (hs.capacity) return DLS_ERR_CAPACITY;
  return hs.corrupt ? DLS_ERR_CORRUPT : DLS_OK;
}

int dls_plan_info(const dls_plan* pl, int32_t* variant, float* tune_ms) {
  if (!pl) return DLS_ERR_INVALID_ARG;
  if (variant) *variant = pl->occ.whole;
  if (tune_ms) { tune_ms[0] = pl->tune_ms[1]; tune_ms[1] = pl->tune_ms[2]; }
  return DLS_OK;
}

int dls_plan_tuning(const dls_plan* pl, int32_t* forms, float* class_ms) {
  if (!pl) return DLS_ERR_INVALID_ARG;
  if (forms) {
    forms[0] = pl->occ.whole;
    forms[1] = pl->occ.rest;
  }
  if (class_ms)
    for (int c = 0; c < 2; ++c)
      for (int f = 0; f < 2; ++f) class_ms[2 * c + f] = pl->class_ms[c][f];
  return DLS_OK;
}

int dls_plan_timing(const dls_plan* pl, float* kernel_ms, int32_t* kernel_nodes) {
  if (!pl) return DLS_ERR_INVALID_ARG;
  if (kernel_nodes) *kernel_nodes = pl->kernel_nodes;
  if (kernel_ms) {
    CK(cudaEventSynchronize(pl->kev[1]));
    CK(cudaEventElapsedTime(kernel_ms, pl->kev[0], pl->kev[1]));
  }
  return DLS_OK;
}

int dls_plan_phase_timing(const dls_plan* pl, float* ms, int32_t count) {
  if (!pl || !ms || count < 6) return DLS_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) ms[i] = 0.0f;
  if (!pl->L.mixed || !pl->exec || !mixed_route(pl->P).tile) return DLS_OK;
  CK(cudaEventSynchronize(pl->pev[4]));
  const cudaEvent_t seq[7] = {pl->kev[0], pl->pev[0], pl->pev[1], pl->pev[2], pl->pev[3], pl->kev[1], pl->pev[4]};
  for (int i = 0; i < 6; ++i) CK(cudaEventElapsedTime(&ms[i], seq[i], seq[i + 1]));
  return DLS_OK;
}

int dls_plan_destroy(dls_plan* pl) {
  if (!pl) return DLS_OK;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->h_status) cudaFreeHost(pl->h_status);
  for (int i = 0; i < 2; ++i)
    if (pl->kev[i]) cudaEventDestroy(pl->kev[i]);
  for (int i = 0; i < 5; ++i)
    if (pl->pev[i]) cudaEventDestroy(pl->pev[i]);
  delete pl;
  return DLS_OK;
}

int dls_phase_cycles(const dls_params* p, const void* d_workspace, unsigned long long* h_cycles, int32_t count) {
  Plan P;
  int st = make_plan(p, &P);
  if (st != DLS_OK) return st;
  const Layout L = work_layout(P);
  if (!L.mixed || !d_workspace || !h_cycles || count < kMixedPhases) return DLS_ERR_INVALID_ARG;
  std::vector<unsigned long long> v((size_t)L.ctas * kMixedPhases);
  CK(cudaMemcpy(v.data(), (const uint8_t*)d_workspace + L.phase, v.size() * sizeof(unsigned long long),
                cudaMemcpyDeviceToHost));
  for (int i = 0; i < kMixedPhases; ++i) h_cycles[i] = 0;
  for (int c = 0; c < L.ctas; ++c)
    for (int i = 0; i < kMixedPhases; ++i) h_cycles[i] += v[(size_t)c * kMixedPhases + i];
  return DLS_OK;
}

int dls_stream_info_get(const void* d_comp, size_t comp_bytes, dls_stream_info* out) {
  if (!out) return DLS_ERR_INVALID_ARG;
  HostHeader h;
  Plan P;
  int st = read_header(d_comp, comp_bytes, 0, &h, &P);
  if (st != DLS_OK) return st;
  memset(out, 0, sizeof(*out));
  out->version = h.version;
  out->nvars = h.p.nvars;
  out->dtype = h.p.dtype;
  out->eb_type = h.p.eb_type;
  out->precision = h.precision;
  out->rank_mode = h.rank_mode;
  out->rank_cap = h.p.rank_cap;
  for (int a = 0; a < 4; ++a) { out->dims[a] = h.p.dims[a]; out->block[a] = h.p.block[a]; }
  out->block_begin = h.p.block_begin;
  out->block_end = h.p.block_end;
  out->total_blocks = h.total_blocks;
  out->total_bytes = (uint64_t)h.total;
  for (int v = 0; v < h.p.nvars; ++v) { out->eb[v] = h.eb[v]; out->delta[v] = h.delta[v]; out->step[v] = h.step[v]; }
  return DLS_OK;
}

int dls_verify(const void* d_orig, const void* d_recon, const void* d_comp, size_t comp_bytes, dls_report* out,
               dls_stream_t stream) {
  if (!d_orig || !d_recon || !out) return DLS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HostHeader h;
  Plan P;
  int st = read_header(d_comp, comp_bytes, s, &h, &P);
  if (st != DLS_OK) return st;
  const size_t nacc = 16 * (size_t)P.nvars + 16;
  double* acc = nullptr;
  CK(cudaMallocAsync((void**)&acc, nacc * sizeof(double), s));
  CK(cudaMemsetAsync(acc, 0, nacc * sizeof(double), s));
  st = launch_verify(P, d_orig, d_recon, d_comp, (unsigned long long)comp_bytes, acc, s);
  std::vector<double> ha(nacc);
  cudaMemcpyAsync(ha.data(), acc, nacc * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(acc, s);
  CK(cudaStreamSynchronize(s));
  if (st != DLS_OK) return st;
  memset(out, 0, sizeof(*out));
  double se = 0, sx = 0;
  int64_t over = 0;
  for (int v = 0; v < P.nvars; ++v) {
    unsigned long long k0, n1;
    memcpy(&k0, &ha[16 * v + 0], 8);
    memcpy(&n1, &ha[16 * v + 1], 8);
    const double mx = k0 ? dunkey(k0) : 0.0;
    out->max_abs_err = fmax(out->max_abs_err, mx);
    over += (int64_t)n1;
    se += ha[16 * v + 2];
    sx += ha[16 * v + 3];
    if (v < 8) {
      out->var_max_abs_err[v] = mx;
      out->var_over[v] = (int64_t)n1;
      out->var_nrmse[v] = ha[16 * v + 3] > 0 ? 100.0 * sqrt(ha[16 * v + 2] / ha[16 * v + 3]) : 0.0;
      out->var_eb[v] = h.eb[v];
    }
  }
  const double* t = &ha[16 * (size_t)P.nvars];
  out->n_over_bound = over;
  out->sum_sq_err = se;
  out->sum_sq = sx;
  out->nrmse = sx > 0 ? 100.0 * sqrt(se / sx) : 0.0;
  out->n_points = P.K * P.nvars;
  out->ratio = (double)(P.K * P.nvars * esize(P.dtype)) / (double)comp_bytes;
  out->n_blocks = P.nb;
  out->n_raw_blocks = (int64_t)t[0];
  out->mean_rank = (P.nb - out->n_raw_blocks) > 0 ? t[1] / (double)(P.nb - out->n_raw_blocks) : 0.0;
  out->n_corr = (int64_t)t[2];
  out->n_esc = (int64_t)t[3];
  out->bytes_basis = (int64_t)t[4];
  out->bytes_coeff = (int64_t)t[5];
  out->bytes_corr = (int64_t)t[6];
  out->bytes_esc = (int64_t)t[7];
  out->bytes_raw = (int64_t)t[8];
  out->bytes_header = (int64_t)t[9] + P.payload_pos;
  if (P.eb_type != DLS_EB_NRMSE && over > 0) return DLS_ERR_BOUND_VIOLATED;
  return DLS_OK;
}

}  // extern "C"
