"""Thin Python binding of the libdls C ABI (include/dls.h).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step of compression, decompression and verification runs
in the library's CUDA kernels.  If libdls.so is not built this module raises;
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

F32, F64 = 0, 1
EB_ABS, EB_REL_RANGE, EB_NRMSE = 0, 1, 2
PREC_FP64, PREC_TF32X3, PREC_BF16X3, PREC_FP32, PREC_TF32, PREC_BF16 = 0, 1, 2, 3, 4, 5
RANK_SEARCH, RANK_LEARNED, RANK_TAIL = 0, 1, 2
MLP_NPARAM, MLP_NFEAT = 6401, 32
OK = 0
ERR_CORRUPT = -4
ERR_TIMEOUT = -6
ERR = {-1: "INVALID_ARG", -2: "CAPACITY", -3: "NONFINITE", -4: "CORRUPT", -5: "CUDA", -6: "TIMEOUT",
       -7: "BOUND_VIOLATED", -8: "WORKSPACE", -9: "NO_MODEL"}


class DlsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {ERR.get(status, status)} ({status})")


class Params(C.Structure):
    _fields_ = [
        ("nvars", C.c_int32),
        ("dims", C.c_int64 * 4),
        ("block", C.c_int32 * 4),
        ("dtype", C.c_int32),
        ("eb_type", C.c_int32),
        ("eb", C.POINTER(C.c_double)),
        ("rank_cap", C.c_int32),
        ("precision", C.c_int32),
        ("rank_mode", C.c_int32),
        ("block_begin", C.c_int64),
        ("block_end", C.c_int64),
        ("basis", C.POINTER(C.c_double)),
        ("basis_n", C.c_int32),
        ("global_stats", C.POINTER(C.c_double)),
        ("corr_codec", C.c_int32),
    ]


class GbParams(C.Structure):
    """dls_gb_params: the global-basis mode's problem (one float32 variable)."""
    _fields_ = [("dims", C.c_int64 * 4), ("m", C.c_int32), ("eps_t", C.c_double), ("nsample", C.c_int64)]


class Report(C.Structure):
    _fields_ = [
        ("max_abs_err", C.c_double), ("n_over_bound", C.c_int64), ("nrmse", C.c_double), ("ratio", C.c_double),
        ("sum_sq_err", C.c_double), ("sum_sq", C.c_double), ("n_points", C.c_int64),
        ("n_blocks", C.c_int64), ("n_raw_blocks", C.c_int64), ("n_corr", C.c_int64), ("n_esc", C.c_int64),
        ("mean_rank", C.c_double),
        ("bytes_header", C.c_int64), ("bytes_basis", C.c_int64), ("bytes_coeff", C.c_int64),
        ("bytes_corr", C.c_int64), ("bytes_esc", C.c_int64), ("bytes_raw", C.c_int64),
        ("var_max_abs_err", C.c_double * 8), ("var_nrmse", C.c_double * 8), ("var_over", C.c_int64 * 8),
        ("var_eb", C.c_double * 8),
    ]


class StreamInfo(C.Structure):
    _fields_ = [
        ("version", C.c_int32), ("nvars", C.c_int32), ("dtype", C.c_int32), ("eb_type", C.c_int32),
        ("precision", C.c_int32), ("rank_mode", C.c_int32), ("rank_cap", C.c_int32),
        ("dims", C.c_int64 * 4), ("block", C.c_int32 * 4),
        ("block_begin", C.c_int64), ("block_end", C.c_int64), ("total_blocks", C.c_int64),
        ("total_bytes", C.c_uint64),
        ("eb", C.c_double * 64), ("delta", C.c_double * 64), ("step", C.c_double * 64),
    ]


_lock = threading.Lock()
_lib = None

# Every symbol include/dls.h declares, with its ctypes signature.
_SIGS = {
    "dls_compress_bound": (C.c_size_t, [C.POINTER(Params)]),
    "dls_workspace_size": (C.c_size_t, [C.POINTER(Params)]),
    "dls_compress": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t),
                               C.c_void_p, C.c_size_t, C.c_void_p]),
    "dls_host_staging_size": (C.c_size_t, [C.POINTER(Params)]),
    "dls_compress_host": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t),
                                    C.c_void_p, C.c_size_t, C.c_void_p]),
    "dls_compress_noalloc": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_size_t,
                                       C.POINTER(C.c_size_t), C.c_void_p]),
    "dls_decompress": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "dls_verify": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(Report), C.c_void_p]),
    "dls_stream_info_get": (C.c_int, [C.c_void_p, C.c_size_t, C.POINTER(StreamInfo)]),
    "dls_set_rank_model": (C.c_int, [C.c_void_p, C.c_size_t]),
    "dls_block_features": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                     C.c_void_p]),
    "dls_field_stats": (C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "dls_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "dls_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dls_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                C.c_int32, C.c_float, C.c_int32, C.c_void_p, C.c_void_p]),
    "dls_plan_create": (C.c_int, [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                                  C.c_void_p, C.POINTER(C.c_void_p)]),
    "dls_plan_execute": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.c_void_p]),
    "dls_plan_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "dls_plan_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "dls_plan_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "dls_plan_destroy": (C.c_int, [C.c_void_p]),
    "dls_plan_phase_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int32]),
    "dls_phase_cycles": (C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_ulonglong), C.c_int32]),
    "dls_stage_quantize": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dls_stage_correct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p]),
    "dls_stage_correct_path": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32, C.c_void_p,
                                         C.c_void_p]),
    "dls_set_fault_hook": (C.c_int, [C.c_int32, C.c_int64]),
    "dls_status_string": (C.c_char_p, [C.c_int]),
    "dls_gb_bound": (C.c_size_t, [C.POINTER(GbParams)]),
    "dls_gb_workspace_size": (C.c_size_t, [C.POINTER(GbParams)]),
    "dls_gb_compress": (C.c_int, [C.POINTER(GbParams), C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.POINTER(C.c_size_t), C.c_void_p, C.c_size_t, C.c_void_p]),
    "dls_gb_decompress": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libdls.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libdls.so is not built ({_build.LIB}); run __graft_entry__.build()")
            L = C.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(st: int) -> str:
    return lib().dls_status_string(st).decode()


def _dtype_code(t: torch.dtype) -> int:
    if t == torch.float32:
        return F32
    if t == torch.float64:
        return F64
    raise TypeError(f"unsupported field dtype {t}")


def make_params(shape, dtype, block, eb, eb_type=EB_ABS, rank_cap=32, precision=PREC_FP64,
                rank_mode=RANK_SEARCH, block_begin=0, block_end=-1, basis=None, global_stats=None, corr_codec=0):
    """shape = (nvars, nt, nz, ny, nx) of the field tensor; basis: optional
    n x n orthonormal modes (column k = mode k) for the blocks of Gram order n;
    global_stats: optional nvars x 4 (min, max, sum of squares, point count) of
    the whole field when the tensor is one part of it (a z-slab): the relative
    bounds and the NRMSE tolerance then come from the whole field; corr_codec:
    1 adds the Rice-coded correction section where it is smaller."""
    nvars, nt, nz, ny, nx = shape
    p = Params()
    p.nvars = nvars
    for a, d in enumerate((nx, ny, nz, nt)):
        p.dims[a] = int(d)
    for a, b in enumerate(block):
        p.block[a] = int(b)
    p.dtype = dtype if isinstance(dtype, int) else _dtype_code(dtype)
    p.eb_type = eb_type
    ebv = [float(eb)] * nvars if not hasattr(eb, "__len__") else [float(e) for e in eb]
    arr = (C.c_double * nvars)(*ebv)
    p.eb = C.cast(arr, C.POINTER(C.c_double))
    p._eb_keep = arr
    p.rank_cap = rank_cap
    p.precision = precision
    p.rank_mode = rank_mode
    p.block_begin = block_begin
    p.block_end = block_end
    p.corr_codec = int(corr_codec)
    if basis is not None:
        import numpy as np
        b = np.ascontiguousarray(np.asarray(basis, dtype=np.float64))
        if b.ndim != 2 or b.shape[0] != b.shape[1]:
            raise ValueError("basis must be a square matrix")
        p.basis = b.ctypes.data_as(C.POINTER(C.c_double))
        p.basis_n = b.shape[0]
        p._basis_keep = b
    if global_stats is not None:
        import numpy as np
        g = np.ascontiguousarray(np.asarray(global_stats, dtype=np.float64))
        if g.shape != (nvars, 4):
            raise ValueError("global_stats must be nvars x 4")
        p.global_stats = g.ctypes.data_as(C.POINTER(C.c_double))
        p._gstats_keep = g
    return p


def compress_bound(p: Params) -> int:
    return lib().dls_compress_bound(C.byref(p))


def workspace_size(p: Params) -> int:
    return lib().dls_workspace_size(C.byref(p))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def compress_into(p: Params, field: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor, stream=None):
    """Raw call: returns (status, nbytes)."""
    nb = C.c_size_t(0)
    st = lib().dls_compress(C.byref(p), C.c_void_p(field.data_ptr()), C.c_void_p(out.data_ptr()), out.numel(),
                            C.byref(nb), C.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream))
    return st, nb.value


def compress(field: torch.Tensor, block, eb, eb_type=EB_ABS, rank_cap=32, precision=PREC_FP64,
             rank_mode=RANK_SEARCH, block_begin=0, block_end=-1, basis=None):
    """Compresses a CUDA field (nvars, nt, nz, ny, nx); returns a uint8 CUDA tensor."""
    if not field.is_cuda or not field.is_contiguous() or field.dim() != 5:
        raise ValueError("field must be a contiguous CUDA tensor (nvars, nt, nz, ny, nx)")
    p = make_params(tuple(field.shape), field.dtype, block, eb, eb_type, rank_cap, precision, rank_mode,
                    block_begin, block_end, basis)
    cap = compress_bound(p)
    ws = workspace_size(p)
    if cap == 0 or ws == 0:
        raise DlsError(-1, "dls_compress")
    out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    work = torch.empty(ws, dtype=torch.uint8, device=field.device)
    st, nb = compress_into(p, field, out, work)
    if st != OK:
        raise DlsError(st, "dls_compress")
    return out[:nb]


def compress_noalloc_into(p: Params, field: torch.Tensor, out: torch.Tensor, stream=None):
    """Compression with the library's built-in 64 MiB workspace, for callers
    that cannot allocate device memory: (status, nbytes)."""
    nb = C.c_size_t(0)
    st = lib().dls_compress_noalloc(C.byref(p), C.c_void_p(field.data_ptr()), C.c_void_p(out.data_ptr()),
                                    out.numel(), C.byref(nb), _stream(stream))
    return st, nb.value


def host_staging_size(p: Params) -> int:
    return lib().dls_host_staging_size(C.byref(p))


def compress_host_into(p: Params, h_field: torch.Tensor, h_out: torch.Tensor, staging: torch.Tensor, stream=None):
    """End-to-end call on host tensors (pinned for full bandwidth): (status, nbytes)."""
    nb = C.c_size_t(0)
    st = lib().dls_compress_host(C.byref(p), C.c_void_p(h_field.data_ptr()), C.c_void_p(h_out.data_ptr()),
                                 h_out.numel(), C.byref(nb), C.c_void_p(staging.data_ptr()), staging.numel(),
                                 _stream(stream))
    return st, nb.value


def stream_info(comp: torch.Tensor) -> StreamInfo:
    info = StreamInfo()
    st = lib().dls_stream_info_get(C.c_void_p(comp.data_ptr()), comp.numel(), C.byref(info))
    if st != OK:
        raise DlsError(st, "dls_stream_info_get")
    return info


def decompress_into(comp: torch.Tensor, out: torch.Tensor, stream=None) -> int:
    return lib().dls_decompress(C.c_void_p(comp.data_ptr()), comp.numel(), C.c_void_p(out.data_ptr()),
                                out.numel() * out.element_size(), _stream(stream))


def decompress(comp: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    if out is None:
        info = stream_info(comp)
        dt = torch.float32 if info.dtype == F32 else torch.float64
        nx, ny, nz, nt = (info.dims[a] for a in range(4))
        out = torch.zeros((info.nvars, nt, nz, ny, nx), dtype=dt, device=comp.device)
    st = decompress_into(comp, out)
    if st != OK:
        raise DlsError(st, "dls_decompress")
    return out


def verify(orig: torch.Tensor, recon: torch.Tensor, comp: torch.Tensor) -> dict:
    rep = Report()
    st = lib().dls_verify(C.c_void_p(orig.data_ptr()), C.c_void_p(recon.data_ptr()), C.c_void_p(comp.data_ptr()),
                          comp.numel(), C.byref(rep), _stream(None))
    if st not in (OK, -7):
        raise DlsError(st, "dls_verify")
    d = {name: getattr(rep, name) for name, _ in Report._fields_}
    for k in ("var_max_abs_err", "var_nrmse", "var_over", "var_eb"):
        d[k] = list(d[k])
    d["status"] = st
    return d


def stage_quantize(c: torch.Tensor, delta: float):
    """Mixed-form quantizer on float32 CUDA coefficients: (q, ovf) int32 tensors."""
    q = torch.empty(c.shape, dtype=torch.int32, device=c.device)
    ovf = torch.empty(c.shape, dtype=torch.int32, device=c.device)
    st = lib().dls_stage_quantize(C.c_void_p(c.data_ptr()), c.numel(), float(delta), C.c_void_p(q.data_ptr()),
                                  C.c_void_p(ovf.data_ptr()), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_stage_quantize")
    return q, ovf


def stage_correct(x: torch.Tensor, xh: torch.Tensor, eb: float):
    """Mixed-form pointwise correction of xh against x (float32 CUDA): int32 k, INT32_MIN = escape."""
    k = torch.empty(x.shape, dtype=torch.int32, device=x.device)
    st = lib().dls_stage_correct(C.c_void_p(x.data_ptr()), C.c_void_p(xh.data_ptr()), x.numel(), float(eb),
                                 C.c_void_p(k.data_ptr()), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_stage_correct")
    return k


CORR_PATH_EXACT, CORR_PATH_SPARSE, CORR_PATH_DENSE = 0, 1, 2
FAULT_NONE, FAULT_WITHHOLD_CHUNK = 0, 1


def stage_correct_path(x: torch.Tensor, xh: torch.Tensor, eb: float, path: int):
    """The pointwise correction through one of the compression's code paths
    (CORR_PATH_*): int32 k, INT32_MIN = escape."""
    k = torch.empty(x.shape, dtype=torch.int32, device=x.device)
    st = lib().dls_stage_correct_path(C.c_void_p(x.data_ptr()), C.c_void_p(xh.data_ptr()), x.numel(), float(eb),
                                      int(path), C.c_void_p(k.data_ptr()), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_stage_correct_path")
    return k


def set_fault_hook(kind: int, arg: int = 0) -> int:
    """Test hook: FAULT_WITHHOLD_CHUNK withholds the first chunk copy of block
    `arg` in later compressions (they return ERR_TIMEOUT); FAULT_NONE clears it."""
    return lib().dls_set_fault_hook(int(kind), int(arg))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def set_rank_model(params) -> None:
    """Loads the block-rank MLP (DLS_MLP_NPARAM float32 values) on the current device."""
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    st = lib().dls_set_rank_model(arr.ctypes.data_as(C.c_void_p), arr.size)
    if st != OK:
        raise DlsError(st, "dls_set_rank_model")


def field_stats(p: Params, field: torch.Tensor, workspace: torch.Tensor | None = None):
    """Per-variable (min, max, sum of squares, points) of a CUDA field as an
    nvars x 4 float64 numpy array (the library's statistics pass)."""
    import numpy as np
    ws = workspace if workspace is not None else torch.empty(workspace_size(p), dtype=torch.uint8,
                                                             device=field.device)
    out = np.zeros((p.nvars, 4), dtype=np.float64)
    st = lib().dls_field_stats(C.byref(p), _ptr(field), out.ctypes.data_as(C.POINTER(C.c_double)), _ptr(ws),
                               ws.numel(), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_field_stats")
    return out


def block_features(field: torch.Tensor, block, eb, eb_type=EB_ABS, rank_cap=16):
    """Per-block features (nb x 32) and bisection ranks (nb) of a float32 CUDA field."""
    p = make_params(tuple(field.shape), field.dtype, block, eb, eb_type, rank_cap, precision=PREC_FP32)
    ws = torch.empty(workspace_size(p), dtype=torch.uint8, device=field.device)
    nb = 1
    for a in range(4):
        nb *= -(-p.dims[a] // p.block[a])
    nb *= p.nvars
    feat = torch.empty((nb, MLP_NFEAT), dtype=torch.float32, device=field.device)
    rank = torch.empty(nb, dtype=torch.int32, device=field.device)
    st = lib().dls_block_features(C.byref(p), _ptr(field), _ptr(feat), _ptr(rank), _ptr(ws), ws.numel(), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_block_features")
    return feat, rank


def mlp_forward(params: torch.Tensor, feat: torch.Tensor) -> torch.Tensor:
    y = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
    st = lib().dls_mlp_forward(_ptr(params), _ptr(feat), feat.shape[0], _ptr(y), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_mlp_forward")
    return y


def mlp_grad(params: torch.Tensor, feat: torch.Tensor, target: torch.Tensor):
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feat.device)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    st = lib().dls_mlp_grad(_ptr(params), _ptr(feat), _ptr(target), feat.shape[0], _ptr(g), _ptr(loss),
                            _stream(None))
    if st != OK:
        raise DlsError(st, "dls_mlp_grad")
    return float(loss.item()), g


def mlp_train(params: torch.Tensor, adam: torch.Tensor, feat: torch.Tensor, target: torch.Tensor,
              order: torch.Tensor, steps: int, batch: int, lr: float, step0: int = 0):
    """Runs `steps` Adam steps on the GPU in place; returns the per-step losses."""
    loss = torch.empty(max(steps, 1), dtype=torch.float32, device=feat.device)
    st = lib().dls_mlp_train(_ptr(params), _ptr(adam), _ptr(feat), _ptr(target), _ptr(order), order.numel(),
                             steps, batch, float(lr), step0, _ptr(loss), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_mlp_train")
    return loss[:steps]


class CompressPlan:
    """Graph-captured, autotuned compression of fixed buffers (dls_plan_*)."""

    def __init__(self, p: Params, field: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor, stream=None):
        self._keep = (p, field, out, workspace)
        self.handle = C.c_void_p()
        st = lib().dls_plan_create(C.byref(p), _ptr(field), _ptr(out), out.numel(), _ptr(workspace),
                                   workspace.numel(), _stream(stream), C.byref(self.handle))
        if st != OK:
            raise DlsError(st, "dls_plan_create")

    def execute(self, stream=None) -> int:
        nb = C.c_size_t(0)
        st = lib().dls_plan_execute(self.handle, C.byref(nb), _stream(stream))
        if st != OK:
            raise DlsError(st, "dls_plan_execute")
        return nb.value

    def info(self):
        v = C.c_int32(0)
        ms = (C.c_float * 2)()
        lib().dls_plan_info(self.handle, C.byref(v), ms)
        return v.value, (ms[0], ms[1])

    def tuning(self) -> dict:
        """The occupancy form per shape class (1: built for 2 CTAs per SM, 2:
        for 4) and each class's device ms in either form while tuning (zeros
        when the choice came from the cache)."""
        forms = (C.c_int32 * 2)()
        ms = (C.c_float * 4)()
        st = lib().dls_plan_tuning(self.handle, forms, ms)
        if st != OK:
            raise DlsError(st, "dls_plan_tuning")
        return {"whole": forms[0], "rest": forms[1], "ms": {"whole": (ms[0], ms[1]), "rest": (ms[2], ms[3])}}

    def timing(self):
        """(device ms of the per-block kernels in the last execute, kernel nodes in the graph)."""
        ms = C.c_float(0.0)
        nk = C.c_int32(0)
        st = lib().dls_plan_timing(self.handle, C.byref(ms), C.byref(nk))
        if st != OK:
            raise DlsError(st, "dls_plan_timing")
        return ms.value, nk.value

    PHASES = ("gram", "eig", "rr", "enc", "tile", "pack")

    def phase_timing(self) -> dict:
        """Device ms of each stage of the last execute (k_gram, k_eig, the
        Rayleigh-Ritz kernels, k_enc, k_tile / k_mixed, scan + record packing)."""
        ms = (C.c_float * 6)()
        st = lib().dls_plan_phase_timing(self.handle, ms, 6)
        if st != OK:
            raise DlsError(st, "dls_plan_phase_timing")
        return {k: ms[i] for i, k in enumerate(self.PHASES)}

    def close(self):
        if self.handle:
            lib().dls_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PHASES = ("gram", "jacobi", "refine", "rayleigh_ritz", "predict", "encode", "decide", "search", "pack",
          "n_accepted", "n_searched", "n_exact_fallback", "tile_wait", "n_tensor_core_gram")


def phase_cycles(p: Params, workspace: torch.Tensor) -> dict:
    """Per-phase cycle counts (summed over CTAs) of the last mixed-form compression."""
    arr = (C.c_ulonglong * len(PHASES))()
    st = lib().dls_phase_cycles(C.byref(p), _ptr(workspace), arr, len(PHASES))
    if st != OK:
        raise DlsError(st, "dls_phase_cycles")
    return {k: int(arr[i]) for i, k in enumerate(PHASES)}


# ---------------------------------------------------------------- global-basis mode
def gb_params(shape, m, eps_t, nsample) -> GbParams:
    """shape = (nt, nz, ny, nx) of one variable."""
    nt, nz, ny, nx = shape
    p = GbParams()
    for a, d in enumerate((nx, ny, nz, nt)):
        p.dims[a] = int(d)
    p.m = int(m)
    p.eps_t = float(eps_t)
    p.nsample = int(nsample)
    return p


def gb_compress(field: torch.Tensor, m: int, eps_t: float, origins) -> torch.Tensor:
    """Global-basis compression of a float32 CUDA variable (nt, nz, ny, nx) with
    the sample patches at `origins` (S x 3 int64, x y z): the DLSG stream as a
    uint8 CUDA tensor."""
    import numpy as np
    if not field.is_cuda or field.dtype != torch.float32 or field.dim() != 4 or not field.is_contiguous():
        raise ValueError("field must be a contiguous float32 CUDA tensor (nt, nz, ny, nx)")
    o = torch.from_numpy(np.ascontiguousarray(np.asarray(origins, dtype=np.int64))).to(field.device)
    p = gb_params(tuple(field.shape), m, eps_t, o.shape[0])
    cap = lib().dls_gb_bound(C.byref(p))
    if cap == 0:
        raise DlsError(-1, "dls_gb_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    ws = torch.empty(lib().dls_gb_workspace_size(C.byref(p)), dtype=torch.uint8, device=field.device)
    nb = C.c_size_t(0)
    st = lib().dls_gb_compress(C.byref(p), _ptr(field), _ptr(o), _ptr(out), out.numel(), C.byref(nb), _ptr(ws),
                               ws.numel(), _stream(None))
    if st != OK:
        raise DlsError(st, "dls_gb_compress")
    return out[:nb.value].clone()


def gb_decompress_into(comp: torch.Tensor, out: torch.Tensor) -> int:
    return lib().dls_gb_decompress(_ptr(comp), comp.numel(), _ptr(out), out.numel(), _stream(None))


def gb_decompress(comp: torch.Tensor) -> torch.Tensor:
    """The variable (nt, nz, ny, nx) in float64 from a DLSG stream."""
    import numpy as np
    h = comp[:80].cpu().numpy()
    nx, ny, nz, nt = (int(v) for v in h[24:56].view(np.uint64))
    out = torch.empty((nt, nz, ny, nx), dtype=torch.float64, device=comp.device)
    st = gb_decompress_into(comp, out)
    if st != OK:
        raise DlsError(st, "dls_gb_decompress")
    return out
