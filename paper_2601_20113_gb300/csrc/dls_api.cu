// Host side of the C ABI: parameter validation, block plan, workspace layout,
// launch sequence and status readback.  See include/dls.h for the contract.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "dls_internal.cuh"

namespace dls {

static int esize(int dtype) { return dtype == DLS_F32 ? 4 : 8; }

// Same rules as the stream decoder applies to headers.
int make_plan(const dls_params* p, Plan* out) {
  if (!p || p->nvars < 1 || p->nvars > kMaxVars || !p->eb) return DLS_ERR_INVALID_ARG;
  if (p->dtype != DLS_F32 && p->dtype != DLS_F64) return DLS_ERR_INVALID_ARG;
  if (p->eb_type < 0 || p->eb_type > 2 || p->rank_cap < 0) return DLS_ERR_INVALID_ARG;
  if (p->precision < 0 || p->precision > 2 || p->rank_mode < 0 || p->rank_mode > 1) return DLS_ERR_INVALID_ARG;
  for (int a = 0; a < 4; ++a)
    if (p->dims[a] < 1 || p->block[a] < 1 || p->block[a] > p->dims[a]) return DLS_ERR_INVALID_ARG;
  const int64_t M = (int64_t)p->block[0] * p->block[1] * p->block[2];
  const int64_t T = p->block[3];
  if ((M < T ? M : T) > kMaxN) return DLS_ERR_INVALID_ARG;
  if (M * T > (1ll << 26)) return DLS_ERR_INVALID_ARG;
  for (int v = 0; v < p->nvars; ++v)
    if (!(p->eb[v] > 0.0) || !isfinite(p->eb[v])) return DLS_ERR_INVALID_ARG;
  Plan P;
  memset(&P, 0, sizeof(P));
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
  size_t meta, vst, q, kc, offsets, vars, status, partial, total;
};

static Layout work_layout(const Plan& P) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (size_t)align_up((int64_t)(off + bytes), 256);
    return o;
  };
  L.meta = take(sizeof(BlockMeta) * (size_t)(P.nb > 0 ? P.nb : 1));
  L.vst = take(sizeof(double) * (size_t)(P.nb > 0 ? P.nb : 1) * P.nmax * P.nmax);
  L.q = take(sizeof(int32_t) * (size_t)(P.pt_count > 0 ? P.pt_count : 1));
  L.kc = take(sizeof(int32_t) * (size_t)(P.pt_count > 0 ? P.pt_count : 1));
  L.offsets = take(sizeof(unsigned long long) * (size_t)(P.nb + 1));
  L.vars = take(sizeof(VarInfo) * kMaxVars);
  L.status = take(sizeof(Status));
  L.partial = take(sizeof(double) * (size_t)stats_partial_doubles(P));
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
  return w;
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
  if (P.precision != DLS_PREC_FP64 || P.rank_mode != DLS_RANK_SEARCH) return DLS_ERR_INVALID_ARG;
  const Layout L = work_layout(P);
  if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace & 255)) return DLS_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(L, d_workspace);
  CK(cudaMemsetAsync(w.status, 0, sizeof(Status), s));
  double* partial = (double*)((uint8_t*)d_workspace + L.partial);
  if ((st = launch_stats_resolve(P, d_in, w, partial, s)) != DLS_OK) return st;
  if ((st = launch_plain_compress(P, d_in, w, s)) != DLS_OK) return st;
  if ((st = launch_scan(P, w, out_cap, d_out, s)) != DLS_OK) return st;
  if ((st = launch_pack(P, d_in, w, d_out, out_cap, s)) != DLS_OK) return st;
  Status hs;
  CK(cudaMemcpyAsync(&hs, w.status, sizeof(Status), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hs.nonfinite) return DLS_ERR_NONFINITE;
  *out_bytes = (size_t)hs.total_bytes;
  if (hs.capacity) return DLS_ERR_CAPACITY;
  return DLS_OK;
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
  CK(cudaMemcpyAsync(base, h_in, inb, cudaMemcpyHostToDevice, s));
  size_t nb = 0;
  st = dls_compress(p, base, base + in, bound, &nb, base + in + out, ws, stream);
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
