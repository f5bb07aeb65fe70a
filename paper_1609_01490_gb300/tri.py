"""Python binding of libtri.so (argument marshalling only).

Every function here has the name of the C entry point it calls (include/tri.h),
takes torch tensors that already live on the GPU, passes their device pointers
and the current CUDA stream through the C ABI, and raises TriError on a
non-zero status.  No step of any computation runs in Python or torch: if the
shared library is missing this module fails to import.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtri.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"libtri.so not found at {_LIB_PATH}: build it first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(_LIB_PATH)

# ------------------------------------------------------------- constants --
TRI_OK, TRI_EINVAL, TRI_ERANGE, TRI_ECUDA, TRI_EOVERFLOW, TRI_ETIMEOUT, TRI_ENOSPACE = range(7)
MAP_LAMBDA, MAP_BB, MAP_RB, MAP_REC, MAP_UTM, MAP_LAMBDA_PDELTA, MAP_TET_TABLE = range(7)
MAP_NAMES = {MAP_LAMBDA: "lambda", MAP_BB: "bb", MAP_RB: "rb", MAP_REC: "rec", MAP_UTM: "utm",
             MAP_LAMBDA_PDELTA: "lambda_pdelta", MAP_TET_TABLE: "tet_table"}
SQRT_X, SQRT_R, SQRT_N = range(3)
FP32, BF16X3, BF16X6 = range(3)
BODY_DUMMY, BODY_SENTINEL, BODY_COUNT = range(3)
LIFE_BIRTH = 1 << 3
LIFE_SURVIVE = (1 << 2) | (1 << 3)
KERNEL_EDM, KERNEL_CA, KERNEL_AT = range(3)
SELECT_FEATURES, SELECT_MAX_CANDIDATES = 14, 18

_u32, _u64, _i32, _sz, _vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
_f32, _f64 = ctypes.c_float, ctypes.c_double
_szp = ctypes.POINTER(ctypes.c_size_t)


class CostModelStruct(ctypes.Structure):
    """tri_cost_model: device parameters, hidden widths, host standardisation."""
    _fields_ = [("theta", _vp), ("h1", _u32), ("h2", _u32), ("mu", ctypes.POINTER(_f64)),
                ("sd", ctypes.POINTER(_f64))]


_SIGS = {
    "tri_status_string": ([_i32], ctypes.c_char_p),
    "tri_version": ([], _i32),
    "tri_map_launch": ([_i32, _i32, _u32, _u32, _i32, _i32, _vp, _vp], _i32),
    "tri_lambda_verify": ([_i32, _i32, _u64, _u64, _vp, _vp], _i32),
    "tri_map_first_error": ([_i32, _i32, _u64, _u64, _u64, _vp, _vp], _i32),
    "tri_peak_probe": ([_i32, _u32, _u32, _vp, _vp, _vp], _i32),
    "tri_edm": ([_vp, _u32, _u32, _vp, _i32, _u32, _u32, _i32, _vp, _sz, _vp, _vp], _i32),
    "tri_edm_workspace_size": ([_u32, _u32, _i32, _szp], _i32),
    "tri_edm_prepare": ([_vp, _u32, _u32, _i32, _vp, _sz, _vp], _i32),
    "tri_edm_gram": ([_u32, _u32, _vp, _i32, _i32, _vp, _sz, _vp], _i32),
    "tri_edm_fixup": ([_vp, _u32, _u32, _vp, _i32, _vp, _sz, _vp, _vp], _i32),
    "tri_edm_host": ([_vp, _u32, _u32, _vp, _i32, _i32, _u32, _vp, _vp, _vp, _sz, _vp, _vp], _i32),
    "tri_edm_partition": ([_u32, _u32, _u32, _vp, _vp, _vp, _vp], _i32),
    "tri_edm_rows": ([_vp, _u32, _u32, _u32, _u32, _vp, _i32, _i32, _vp, _sz, _vp, _vp], _i32),
    "tri_edm_batched": ([_vp, _vp, _vp, _u32, _u32, _vp, _vp, _u32, _u32, _vp, _sz, _vp], _i32),
    "tri_edm_batched_workspace_size": ([_u32, _szp], _i32),
    "tri_edm_batched_partition": ([_vp, _u32, _u32, _u32, _u32, _u32, _vp, _vp], _i32),
    "tri_ca_step": ([_vp, _vp, _u32, _sz, _u32, _u32, _i32, _u32, _vp], _i32),
    "tri_ca_run": ([_vp, _vp, _vp, _u32, _sz, _u32, _u32, _i32, _u32, _u32, _vp], _i32),
    "tri_ca_partition": ([_u32, _u32, _u32, _u32, _vp, _vp], _i32),
    "tri_ca_step_rows": ([_vp, _vp, _u32, _sz, _u32, _u32, _u32, _u32, _u32, _vp], _i32),
    "tri_collide": ([_vp, _vp, _u32, _u32, _i32, _u32, _u32, _vp, _vp, _u64, _vp, _vp], _i32),
    "tet_map": ([_u32, _u32, _i32, _vp, _vp], _i32),
    "tet_map_ex": ([_i32, _u32, _u32, _i32, _vp, _vp], _i32),
    "tet_at_energy": ([_vp, _u32, _f64, _vp, _i32, _u32, _vp, _sz, _vp], _i32),
    "tet_at_workspace_size": ([_u32, _u32, _i32, _szp], _i32),
    "tet_at_energy_noalloc": ([_vp, _u32, _f64, _vp, _i32, _u32, _vp], _i32),
    "tet_at_partition": ([_u32, _u32, _u32, _u32, _vp, _vp], _i32),
    "tet_at_energy_range": ([_vp, _u32, _f64, _vp, _i32, _u32, _u64, _u64, _vp, _sz, _vp], _i32),
    "tri_mlp_workspace_size": ([_u32, _u32, _u32, _szp], _i32),
    "tri_mlp_forward": ([_vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _sz, _vp], _i32),
    "tri_mlp_grad": ([_vp, _vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _vp, _sz, _vp], _i32),
    "tri_mlp_adam": ([_vp, _vp, _vp, _vp, _u32, _u32, _f32, _f32, _f32, _f32, _vp], _i32),
    "tri_mlp_argmin": ([_vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _sz, _vp], _i32),
    "tri_select_features": ([_i32, _u32, _u32, _vp, _vp, _vp, _vp], _i32),
    "tri_select_workspace_size": ([_u32, _u32, _szp], _i32),
    "tri_select": ([ctypes.POINTER(CostModelStruct), _i32, _u32, _u32, _vp, _vp, _vp, _sz, _vp], _i32),
    "tri_sync_status": ([_vp, _vp, _vp], _i32),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

LIB_PATH = _LIB_PATH
EXPORTS = tuple(_SIGS)


class TriError(RuntimeError):
    def __init__(self, call: str, status: int):
        super().__init__(f"{call}: {_lib.tri_status_string(status).decode()} (status {status})")
        self.status = status


def _check(call: str, st: int) -> None:
    if st != TRI_OK:
        raise TriError(call, st)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def _hptr(t) -> int:
    """Pointer of a contiguous host (CPU) tensor; pinned memory keeps the copies asynchronous."""
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _size(fn, *args) -> int:
    out = ctypes.c_size_t(0)
    _check(fn.__name__, fn(*args, ctypes.byref(out)))
    return int(out.value)


def tri_version() -> int:
    return int(_lib.tri_version())


# ------------------------------------------------------------------ maps --
def tri_map_launch(map: int, sqrt_kind: int, n: int, rho: int, with_diag: bool, body: int, out,
                   stream=None) -> None:
    _check("tri_map_launch", _lib.tri_map_launch(map, sqrt_kind, n, rho, 1 if with_diag else 0, body,
                                                 _ptr(out), _stream(stream)))


def tri_peak_probe(kind: int, blocks: int, iters: int, sink, stream=None) -> float:
    """Launches the FMA probe; returns the flop it performs (the caller times it)."""
    flop = ctypes.c_double(0.0)
    _check("tri_peak_probe", _lib.tri_peak_probe(kind, blocks, iters, _ptr(sink), ctypes.addressof(flop),
                                                 _stream(stream)))
    return flop.value


def tri_map_first_error(map: int, sqrt_kind: int, n_items: int, begin: int, end: int, first_bad,
                        stream=None) -> None:
    _check("tri_map_first_error", _lib.tri_map_first_error(map, sqrt_kind, n_items, begin, end, _ptr(first_bad),
                                                           _stream(stream)))


def tri_lambda_verify(sqrt_kind: int, with_diag: bool, w_begin: int, w_end: int, result, stream=None) -> None:
    _check("tri_lambda_verify", _lib.tri_lambda_verify(sqrt_kind, 1 if with_diag else 0, w_begin, w_end,
                                                       _ptr(result), _stream(stream)))


def tet_map(n: int, rho: int, body: int, out, stream=None) -> None:
    _check("tet_map", _lib.tet_map(n, rho, body, _ptr(out), _stream(stream)))


def tet_map_ex(map: int, n: int, rho: int, body: int, out, stream=None) -> None:
    _check("tet_map_ex", _lib.tet_map_ex(map, n, rho, body, _ptr(out), _stream(stream)))


# ------------------------------------------------------------------- EDM --
def tri_edm_workspace_size(n: int, d: int, prec: int) -> int:
    return _size(_lib.tri_edm_workspace_size, n, d, prec)


def tri_edm(x, out, map: int = MAP_LAMBDA, rho: int = 16, reg: int = 0, prec: int = FP32, workspace=None,
            n_flagged=None, stream=None) -> None:
    n, d = x.shape
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("tri_edm", _lib.tri_edm(_ptr(x), n, d, _ptr(out), map, rho, reg, prec, _ptr(workspace), ws_bytes,
                                   _ptr(n_flagged), _stream(stream)))


def tri_edm_host(x_host, out_host, x_dev, out_dev, workspace, map: int = MAP_LAMBDA, prec: int = BF16X6,
                 bands: int = 0, n_flagged=None, stream=None) -> None:
    """Host buffers in and out (pinned CPU tensors), device buffers and workspace
    supplied by the caller; the call enqueues the work on `stream`."""
    n, d = x_host.shape
    ws_bytes = workspace.numel() * workspace.element_size()
    _check("tri_edm_host", _lib.tri_edm_host(_hptr(x_host), n, d, _hptr(out_host), map, prec, bands, _ptr(x_dev),
                                             _ptr(out_dev), _ptr(workspace), ws_bytes, _ptr(n_flagged),
                                             _stream(stream)))


def _nbytes(t) -> int:
    return t.numel() * t.element_size() if t is not None else 0


def tri_edm_prepare(x, prec: int, workspace, stream=None) -> None:
    n, d = x.shape
    _check("tri_edm_prepare", _lib.tri_edm_prepare(_ptr(x), n, d, prec, _ptr(workspace), _nbytes(workspace),
                                                   _stream(stream)))


def tri_edm_gram(n: int, d: int, out, map: int, prec: int, workspace, stream=None) -> None:
    _check("tri_edm_gram", _lib.tri_edm_gram(n, d, _ptr(out), map, prec, _ptr(workspace), _nbytes(workspace),
                                             _stream(stream)))


def tri_edm_fixup(x, out, prec: int, workspace, n_flagged=None, stream=None) -> None:
    n, d = x.shape
    _check("tri_edm_fixup", _lib.tri_edm_fixup(_ptr(x), n, d, _ptr(out), prec, _ptr(workspace),
                                               _nbytes(workspace), _ptr(n_flagged), _stream(stream)))


def tri_edm_partition(n: int, ranks: int, rank: int):
    """(row_begin, row_end, pair_begin, pair_end) of rank `rank` of `ranks` (host only)."""
    rb, re_, pb, pe = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    _check("tri_edm_partition", _lib.tri_edm_partition(n, ranks, rank, ctypes.byref(rb), ctypes.byref(re_),
                                                       ctypes.byref(pb), ctypes.byref(pe)))
    return rb.value, re_.value, pb.value, pe.value


def tri_edm_rows(x, row_begin: int, row_end: int, out_band, map: int = MAP_LAMBDA, prec: int = BF16X6,
                 workspace=None, n_flagged=None, stream=None) -> None:
    n, d = x.shape
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("tri_edm_rows", _lib.tri_edm_rows(_ptr(x), n, d, row_begin, row_end, _ptr(out_band), map, prec,
                                             _ptr(workspace), ws_bytes, _ptr(n_flagged), _stream(stream)))


def tri_edm_batched_workspace_size(count: int) -> int:
    return _size(_lib.tri_edm_batched_workspace_size, count)


def tri_edm_batched(x_cat, pt_off, n_k, out_cat, out_off, rho: int = 16, reg: int = 0, workspace=None,
                    stream=None) -> None:
    count = n_k.numel()
    d = x_cat.shape[1]
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("tri_edm_batched", _lib.tri_edm_batched(_ptr(x_cat), _ptr(pt_off), _ptr(n_k), count, d,
                                                   _ptr(out_cat), _ptr(out_off), rho, reg, _ptr(workspace),
                                                   ws_bytes, _stream(stream)))


def tri_edm_batched_partition(n_k_host, rho: int, reg: int, ranks: int, rank: int):
    """(k_begin, k_end): the instances rank `rank` of `ranks` computes (host only;
    n_k_host: the instance sizes as a sequence or a host array)."""
    import numpy as np
    nk = np.ascontiguousarray(np.asarray(n_k_host, dtype=np.uint32))
    kb, ke = ctypes.c_uint32(), ctypes.c_uint32()
    _check("tri_edm_batched_partition",
           _lib.tri_edm_batched_partition(nk.ctypes.data if nk.size else None, nk.size, rho, reg, ranks, rank,
                                          ctypes.byref(kb), ctypes.byref(ke)))
    return kb.value, ke.value


# -------------------------------------------------------------------- CA --
def tri_collide(centres, radii, n_pairs, count=None, pairs=None, map: int = MAP_LAMBDA, rho: int = 16,
                reg: int = 0, stream=None) -> None:
    """Collision detection of the spheres (centres [n][dim] FP32, radii [n]):
    n_pairs (uint64 [1]) gets the number of colliding pairs, count (int32 or
    uint32 [n]) the per-sphere counts, pairs (int32 or uint32 [cap][2]) the
    first cap pairs (i, j), i > j, in no particular order."""
    n = centres.shape[0]
    dim = centres.shape[1] if centres.dim() == 2 else 1
    cap = pairs.shape[0] if pairs is not None else 0
    _check("tri_collide", _lib.tri_collide(_ptr(centres), _ptr(radii), n, dim, map, rho, reg, _ptr(count),
                                           _ptr(pairs), cap, _ptr(n_pairs), _stream(stream)))


def tri_ca_step(inp, out, n: int, birth_mask: int = LIFE_BIRTH, survive_mask: int = LIFE_SURVIVE,
                map: int = MAP_LAMBDA, rho: int = 16, stream=None) -> None:
    ld = inp.stride(0)
    if out.stride(0) != ld:
        raise ValueError("in and out must share the leading dimension")
    _check("tri_ca_step", _lib.tri_ca_step(_ptr(inp), _ptr(out), n, ld, birth_mask, survive_mask, map, rho,
                                           _stream(stream)))


def tri_ca_run(inp, out, n: int, steps: int, scratch=None, birth_mask: int = LIFE_BIRTH,
               survive_mask: int = LIFE_SURVIVE, map: int = MAP_LAMBDA, rho: int = 32, stream=None) -> None:
    ld = inp.stride(0)
    if out.stride(0) != ld or (scratch is not None and scratch.stride(0) != ld):
        raise ValueError("in, out and scratch must share the leading dimension")
    _check("tri_ca_run", _lib.tri_ca_run(_ptr(inp), _ptr(out), _ptr(scratch), n, ld, birth_mask, survive_mask, map,
                                         rho, steps, _stream(stream)))


def tri_ca_partition(n: int, rho: int, ranks: int, rank: int):
    """(row_begin, row_end) of rank `rank` of `ranks` (host only)."""
    rb, re_ = ctypes.c_uint32(), ctypes.c_uint32()
    _check("tri_ca_partition", _lib.tri_ca_partition(n, rho, ranks, rank, ctypes.byref(rb), ctypes.byref(re_)))
    return rb.value, re_.value


def tri_ca_step_rows(inp, out, n: int, row_begin: int, row_end: int, birth_mask: int = LIFE_BIRTH,
                     survive_mask: int = LIFE_SURVIVE, rho: int = 32, stream=None) -> None:
    ld = inp.stride(0)
    if out.stride(0) != ld:
        raise ValueError("in and out must share the leading dimension")
    _check("tri_ca_step_rows", _lib.tri_ca_step_rows(_ptr(inp), _ptr(out), n, ld, birth_mask, survive_mask, rho,
                                                     row_begin, row_end, _stream(stream)))


# -------------------------------------------------------------------- AT --
def tet_at_workspace_size(n: int, rho: int, map: int = MAP_LAMBDA) -> int:
    return _size(_lib.tet_at_workspace_size, n, rho, map)


def tet_at_energy(xyz, energy, nu: float = 1.0, map: int = MAP_LAMBDA, rho: int = 16, workspace=None,
                  stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("tet_at_energy", _lib.tet_at_energy(_ptr(xyz), xyz.shape[0], float(nu), _ptr(energy), map, rho,
                                               _ptr(workspace), ws_bytes, _stream(stream)))


def tet_at_energy_noalloc(xyz, energy, nu: float = 1.0, map: int = MAP_LAMBDA, rho: int = 16,
                          stream=None) -> None:
    """tet_at_energy with its scratch in an array inside the library, for
    callers that cannot allocate device memory (see include/tri.h)."""
    _check("tet_at_energy_noalloc", _lib.tet_at_energy_noalloc(_ptr(xyz), xyz.shape[0], float(nu), _ptr(energy),
                                                               map, rho, _stream(stream)))


def tet_at_partition(n: int, rho: int, ranks: int, rank: int):
    """(omega_begin, omega_end) of rank `rank` of `ranks` (host only)."""
    w0, w1 = ctypes.c_uint64(), ctypes.c_uint64()
    _check("tet_at_partition", _lib.tet_at_partition(n, rho, ranks, rank, ctypes.byref(w0), ctypes.byref(w1)))
    return w0.value, w1.value


def tet_at_energy_range(xyz, energy, omega_begin: int, omega_end: int, nu: float = 1.0, map: int = MAP_LAMBDA,
                        rho: int = 32, workspace=None, stream=None) -> None:
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("tet_at_energy_range", _lib.tet_at_energy_range(_ptr(xyz), xyz.shape[0], float(nu), _ptr(energy), map,
                                                           rho, omega_begin, omega_end, _ptr(workspace), ws_bytes,
                                                           _stream(stream)))


# ------------------------------------------------------------------- MLP --
def tri_mlp_workspace_size(B: int, H1: int, H2: int) -> int:
    return _size(_lib.tri_mlp_workspace_size, B, H1, H2)


def _ws(workspace):
    return _ptr(workspace), workspace.numel() * workspace.element_size()


def tri_mlp_forward(theta, X, pred, H1: int, H2: int, workspace, stream=None) -> None:
    B, F = X.shape
    p, nb = _ws(workspace)
    _check("tri_mlp_forward", _lib.tri_mlp_forward(_ptr(theta), _ptr(X), B, F, H1, H2, _ptr(pred), p, nb,
                                                   _stream(stream)))


def tri_mlp_grad(theta, X, y, loss, grad, H1: int, H2: int, workspace, stream=None) -> None:
    B, F = X.shape
    p, nb = _ws(workspace)
    _check("tri_mlp_grad", _lib.tri_mlp_grad(_ptr(theta), _ptr(X), _ptr(y), B, F, H1, H2, _ptr(loss),
                                             _ptr(grad), p, nb, _stream(stream)))


def tri_mlp_adam(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, stream=None) -> None:
    _check("tri_mlp_adam", _lib.tri_mlp_adam(_ptr(theta), _ptr(grad), _ptr(m), _ptr(v), theta.numel(), t, lr,
                                             beta1, beta2, eps, _stream(stream)))


def tri_mlp_argmin(theta, X, best, H1: int, H2: int, workspace, stream=None) -> None:
    B, F = X.shape
    p, nb = _ws(workspace)
    _check("tri_mlp_argmin", _lib.tri_mlp_argmin(_ptr(theta), _ptr(X), B, F, H1, H2, _ptr(best), p, nb,
                                                 _stream(stream)))


def tri_select_features(kernel: int, n: int, d: int):
    """Host only: (X [count][14] FP32 raw features, maps, rhos) of the candidates."""
    import numpy as np
    X = np.zeros((SELECT_MAX_CANDIDATES, SELECT_FEATURES), dtype=np.float32)
    maps = np.zeros(SELECT_MAX_CANDIDATES, dtype=np.int32)
    rhos = np.zeros(SELECT_MAX_CANDIDATES, dtype=np.uint32)
    count = ctypes.c_uint32(0)
    _check("tri_select_features", _lib.tri_select_features(kernel, n, d, X.ctypes.data, maps.ctypes.data,
                                                           rhos.ctypes.data, ctypes.addressof(count)))
    c = count.value
    return X[:c].copy(), [int(v) for v in maps[:c]], [int(v) for v in rhos[:c]]


def tri_select_workspace_size(h1: int, h2: int) -> int:
    return _size(_lib.tri_select_workspace_size, h1, h2)


def tri_select(theta, h1: int, h2: int, mu, sd, kernel: int, n: int, d: int, workspace, stream=None):
    """(map, rho) picked by the cost model (theta on the device, mu and sd host
    FP64 arrays); theta None gives the library default.  Synchronises the stream."""
    import numpy as np
    mu64 = np.ascontiguousarray(mu, dtype=np.float64)
    sd64 = np.ascontiguousarray(sd, dtype=np.float64)
    model = CostModelStruct(_ptr(theta) if theta is not None else None, h1, h2,
                            mu64.ctypes.data_as(ctypes.POINTER(_f64)), sd64.ctypes.data_as(ctypes.POINTER(_f64)))
    m, r = ctypes.c_int(0), ctypes.c_uint32(0)
    p, nb = _ws(workspace)
    _check("tri_select", _lib.tri_select(ctypes.byref(model), kernel, n, d, ctypes.addressof(m),
                                         ctypes.addressof(r), p, nb, _stream(stream)))
    return m.value, r.value


def tri_sync_status(status, stream=None) -> int:
    """Synchronise the stream and read one device status word (an int32 tensor element)."""
    v = ctypes.c_int(0)
    _check("tri_sync_status", _lib.tri_sync_status(_ptr(status), ctypes.addressof(v), _stream(stream)))
    return v.value
