"""Python binding of libdmrg2d (include/dmrg2d.h): argument marshalling only.

Every step of the H·v path and the solvers runs in the library's CUDA kernels;
this module converts numpy/torch arguments into the C structures and device
pointers.  There is no fallback: if the shared library is missing or fails to
load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HEISENBERG, HUBBARD = 0, 1
FP64, TF32, BF16, FP32, FP64X, BF16X3 = 0, 1, 2, 3, 4, 5
PRECISION = {"fp64": FP64, "tf32": TF32, "bf16": BF16, "fp32": FP32, "fp64x": FP64X,
             "bf16x3": BF16X3}
STATUS = {0: "OK", -1: "EINVAL", -2: "ESHAPE", -3: "ENOMEM", -4: "ECUDA", -5: "ENOCONV",
          -6: "ETIMEOUT", -7: "ENAN", -8: "EUNSUPPORTED"}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdmrg2d.so")
_lib = None


class Dmrg2dError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_legs", C.c_int), ("J_leg", C.c_double),
                ("J_rung", C.c_double), ("t", C.c_double), ("U", C.c_double), ("rung_pbc", C.c_int)]


class Block(C.Structure):
    _fields_ = [("m", C.c_int), ("H", C.POINTER(C.c_double)), ("n_edge", C.c_int),
                ("edge", C.POINTER(C.POINTER(C.c_double))), ("parity", C.POINTER(C.c_double)),
                ("qn", C.POINTER(C.c_int32))]


class SweepOpts(C.Structure):
    _fields_ = [("n_columns", C.c_int), ("m_warmup", C.c_int), ("n_sweeps", C.c_int),
                ("m_sweep", C.POINTER(C.c_int)), ("precision", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("krylov_dim", C.c_int), ("seed", C.c_uint64),
                ("use_sectors", C.c_int), ("n_up", C.c_int), ("n_dn", C.c_int),
                ("solver", C.c_int), ("precond", C.c_int), ("mlp", C.c_void_p),
                ("mlp_train_sweeps", C.c_int), ("mlp_epochs", C.c_int)]


class SweepReport(C.Structure):
    _fields_ = [("cap", C.c_int), ("n_steps", C.c_int), ("energy", C.POINTER(C.c_double)),
                ("trunc", C.POINTER(C.c_double)), ("l", C.POINTER(C.c_int)),
                ("sweep", C.POINTER(C.c_int)), ("iters", C.POINTER(C.c_int)),
                ("leg_bond", C.POINTER(C.c_double)), ("rung_bond", C.POINTER(C.c_double)),
                ("s2", C.POINTER(C.c_double)), ("densities", C.POINTER(C.c_double)),
                ("seconds", C.c_double),
                ("solve_seconds", C.c_double), ("build_seconds", C.c_double),
                ("dm_seconds", C.c_double), ("renorm_seconds", C.c_double),
                ("obs_seconds", C.c_double), ("train_seconds", C.c_double),
                ("transform_seconds", C.c_double)]


class StateInfo(C.Structure):
    _fields_ = [("n_columns", C.c_int), ("warmed_up", C.c_int), ("sweeps_done", C.c_int),
                ("last_energy", C.c_double), ("m_left", C.c_int), ("m_right", C.c_int),
                ("failed", C.c_int)]


class OpsInfo(C.Structure):
    _fields_ = [("n_vec", C.c_int64), ("m1", C.c_int), ("m4", C.c_int), ("d", C.c_int),
                ("n_legs", C.c_int), ("n_blk_left", C.c_int), ("n_blk_right", C.c_int),
                ("n_scalar", C.c_int), ("flops_per_apply", C.c_double), ("tc_ok", C.c_int),
                ("device_bytes", C.c_int64), ("n_sectors", C.c_int)]


class SolverOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("krylov_dim", C.c_int), ("tol", C.c_double),
                ("fixed_steps", C.c_int), ("precision", C.c_int), ("refine", C.c_int),
                ("inner_iter", C.c_int), ("outer_max", C.c_int), ("check_every", C.c_int),
                ("start_reorth", C.c_int), ("refine_precision", C.c_int),
                ("thick_keep", C.c_int)]


class DavidsonOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("max_subspace", C.c_int), ("tol", C.c_double),
                ("precision", C.c_int), ("refine", C.c_int), ("precond", C.c_int),
                ("mlp", C.c_void_p), ("inner_iter", C.c_int), ("outer_max", C.c_int),
                ("refine_tol", C.c_double), ("log_cap", C.c_int), ("log_x", C.c_void_p),
                ("log_r", C.c_void_p), ("log_theta", C.POINTER(C.c_double))]


class SolverStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("n_hv_fp64", C.c_int),
                ("n_hv_low", C.c_int), ("resid", C.c_double), ("hv_ms", C.c_double),
                ("elapsed_ms", C.c_double)]


# every symbol include/dmrg2d.h declares, with its ctypes signature
SIGNATURES = {
    "dmrg2d_build_ops": (C.c_int, [C.POINTER(Model), C.POINTER(Block), C.POINTER(Block),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_void_p), C.c_void_p]),
    "dmrg2d_ops_get_info": (C.c_int, [C.c_void_p, C.POINTER(OpsInfo)]),
    "dmrg2d_sector_dense_index": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dmrg2d_apply_H": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dmrg2d_convert_input": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_void_p]),
    "dmrg2d_lanczos_ground": (C.c_int, [C.c_void_p, C.POINTER(SolverOpts), C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(SolverStats), C.c_void_p]),
    "dmrg2d_lanczos_ground_noalloc": (C.c_int, [C.c_void_p, C.POINTER(SolverOpts), C.c_void_p,
                                                C.POINTER(C.c_double), C.POINTER(SolverStats),
                                                C.c_void_p]),
    "dmrg2d_default_solver_opts": (None, [C.POINTER(SolverOpts)]),
    "dmrg2d_tridiag_lowest": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "dmrg2d_wait_selftest": (C.c_int, [C.c_double, C.c_void_p]),
    "dmrg2d_sweep": (C.c_int, [C.c_void_p, C.POINTER(SweepOpts), C.POINTER(SweepReport),
                               C.c_void_p]),
    "dmrg2d_state_create": (C.c_int, [C.POINTER(Model), C.POINTER(SweepOpts),
                                      C.POINTER(C.c_void_p)]),
    "dmrg2d_state_free": (None, [C.c_void_p]),
    "dmrg2d_state_get_info": (C.c_int, [C.c_void_p, C.POINTER(StateInfo)]),
    "dmrg2d_diagonal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg2d_default_davidson_opts": (None, [C.POINTER(DavidsonOpts)]),
    "dmrg2d_davidson_ground": (C.c_int, [C.c_void_p, C.POINTER(DavidsonOpts), C.c_void_p,
                                         C.POINTER(C.c_double), C.POINTER(SolverStats),
                                         C.c_void_p]),
    "dmrg2d_mlp_create": (C.c_int, [C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    "dmrg2d_mlp_free": (None, [C.c_void_p]),
    "dmrg2d_mlp_num_params": (C.c_int, [C.c_void_p]),
    "dmrg2d_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dmrg2d_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dmrg2d_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "dmrg2d_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                       C.c_void_p, C.POINTER(C.c_float), C.c_void_p]),
    "dmrg2d_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                        C.c_float, C.POINTER(C.c_float), C.c_void_p]),
    "dmrg2d_mlp_make_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg2d_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_int,
                                  C.c_void_p]),
    "dmrg2d_set_tile_config": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "dmrg2d_tile_config_name": (C.c_char_p, [C.c_int]),
    "dmrg2d_free_ops": (None, [C.c_void_p]),
    "dmrg2d_check_device": (C.c_int, [C.c_void_p]),
    "dmrg2d_profile_start": (C.c_int, [C.c_void_p, C.c_int]),
    "dmrg2d_profile_stop": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "dmrg2d_site_densities": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dmrg2d_last_error": (C.c_char_p, []),
    "dmrg2d_version": (C.c_char_p, []),
    "dmrg2d_struct_size": (C.c_size_t, [C.c_int]),
}


def lib():
    """Load libdmrg2d.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} not built: run paper_0707_0159_gb300.build.build()")
        h = C.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def last_error() -> str:
    return lib().dmrg2d_last_error().decode()


def version() -> str:
    return lib().dmrg2d_version().decode()


def _check(code):
    if code != 0:
        raise Dmrg2dError(code, last_error())


def _stream(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():   # argument checks still run; device calls fail
            return C.c_void_p(0)
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class _BlockArgs:
    """Keeps the numpy buffers of one block alive while the C struct points at them."""

    def __init__(self, blk: dict, nq: int):
        m = int(blk["m"])
        self.H = np.ascontiguousarray(blk["H"], dtype=np.float64).reshape(m, m)
        self.edge = [np.ascontiguousarray(e, dtype=np.float64).reshape(m, m) for e in blk["edge"]]
        self.ptrs = (C.POINTER(C.c_double) * max(1, len(self.edge)))(
            *[e.ctypes.data_as(C.POINTER(C.c_double)) for e in self.edge])
        par = blk.get("parity")
        self.par = None if par is None else np.ascontiguousarray(par, dtype=np.float64).reshape(m)
        qn = blk.get("qn")
        self.qn = None if qn is None else np.ascontiguousarray(qn, dtype=np.int32).reshape(m, nq)
        self.c = Block(
            m, self.H.ctypes.data_as(C.POINTER(C.c_double)), len(self.edge),
            self.ptrs if self.edge else None,
            None if self.par is None else self.par.ctypes.data_as(C.POINTER(C.c_double)),
            None if self.qn is None else self.qn.ctypes.data_as(C.POINTER(C.c_int32)))


class Ops:
    """Owner of a dmrg2d_ops* (freed with the object)."""

    def __init__(self, ptr):
        self._p = ptr
        inf = OpsInfo()
        _check(lib().dmrg2d_ops_get_info(ptr, C.byref(inf)))
        self.info = {k: getattr(inf, k) for k, _ in OpsInfo._fields_}

    @property
    def ptr(self):
        return self._p

    def free(self):
        if self._p:
            lib().dmrg2d_free_ops(self._p)
            self._p = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _model(model: dict) -> Model:
    kind = HEISENBERG if model["kind"] == "heisenberg" else HUBBARD
    return Model(kind, int(model["n_legs"]), float(model.get("J_leg", 1.0)),
                 float(model.get("J_rung", 1.0)), float(model.get("t", 1.0)),
                 float(model.get("U", 0.0)), int(bool(model.get("rung_pbc", False))))


def build_ops(model: dict, left: dict, right: dict, target=None, stream=None) -> Ops:
    mdl = _model(model)
    nq = 1 if mdl.kind == HEISENBERG else 2
    la, ra = _BlockArgs(left, nq), _BlockArgs(right, nq)
    tgt = None
    if target is not None:
        tgt = (C.c_int32 * nq)(*[int(x) for x in target])
    out = C.c_void_p()
    code = lib().dmrg2d_build_ops(C.byref(mdl), C.byref(la.c), C.byref(ra.c), tgt, C.byref(out),
                                  _stream(stream))
    _check(code)
    return Ops(out)


def sector_dense_index(ops: Ops) -> np.ndarray:
    """Dense superblock index of every packed position (-1 for padding rows)."""
    out = np.empty(ops.info["n_vec"], dtype=np.int64)
    _check(lib().dmrg2d_sector_dense_index(ops.ptr, out.ctypes.data_as(C.c_void_p)))
    return out


_DTYPES = {FP64: ("float64", "float64"), FP32: ("float32", "float32"),
           TF32: ("float32", "float32"), BF16: ("bfloat16", "float32"),
           FP64X: ("float64", "float64"), BF16X3: ("bfloat16", "float32")}
_IN_PARTS = {BF16X3: 2}   # BF16X3 input: hi part then lo part


def apply_H(ops: Ops, v, y, precision=FP64, stream=None):
    """y = H v on the device (torch CUDA tensors, contiguous, n_vec elements; the BF16X3
    input holds 2 n_vec elements, see convert_input)."""
    precision = PRECISION.get(precision, precision)
    vin, vout = _DTYPES[precision]
    n = ops.info["n_vec"]
    for t, dt, name, cnt in ((v, vin, "v", n * _IN_PARTS.get(precision, 1)), (y, vout, "y", n)):
        if not t.is_cuda or not t.is_contiguous() or t.numel() != cnt or str(t.dtype) != "torch." + dt:
            raise ValueError(f"{name}: need a contiguous CUDA {dt} tensor of {cnt} elements, got "
                             f"{t.dtype} {tuple(t.shape)} on {t.device}")
    _check(lib().dmrg2d_apply_H(ops.ptr, C.c_void_p(v.data_ptr()), C.c_void_p(y.data_ptr()),
                                int(precision), _stream(stream)))


def convert_input(x, precision, stream=None):
    """The apply_H input at `precision` from the CUDA float64 tensor x
    (dmrg2d_convert_input); returns a new tensor (2 x.numel() bf16 values for BF16X3)."""
    import torch
    precision = PRECISION.get(precision, precision)
    if not x.is_cuda or str(x.dtype) != "torch.float64" or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA float64 tensor")
    # an unknown precision is passed on for the library to reject (EINVAL)
    dt = getattr(torch, _DTYPES.get(precision, ("float64", "float64"))[0])
    out = torch.empty(x.numel() * _IN_PARTS.get(precision, 1), dtype=dt, device=x.device)
    _check(lib().dmrg2d_convert_input(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                      int(precision), int(x.numel()), _stream(stream)))
    return out


def wait_selftest(seconds: float = 0.05, stream=None) -> int:
    """Run the bounded-wait self-test; returns its status code (ETIMEOUT = -6 expected)."""
    return lib().dmrg2d_wait_selftest(float(seconds), _stream(stream))


def check_device(ops: Ops):
    """Raise if a device-side bounded wait gave up since the last check."""
    _check(lib().dmrg2d_check_device(ops.ptr))


def profile_start(ops: Ops, max_launches: int):
    _check(lib().dmrg2d_profile_start(ops.ptr, int(max_launches)))


def profile_stop(ops: Ops):
    """(summed dominant-kernel milliseconds, timed launches) since profile_start."""
    ms, n = C.c_double(), C.c_int()
    _check(lib().dmrg2d_profile_stop(ops.ptr, C.byref(ms), C.byref(n)))
    return ms.value, n.value


N_TILE_CONFIGS = 27


def autotune(ops: Ops, precision, stream=None):
    """Time every tensor-core tile configuration; keep the fastest. Returns (best, ms list)."""
    precision = PRECISION.get(precision, precision)
    ms = (C.c_double * N_TILE_CONFIGS)()
    best = C.c_int()
    _check(lib().dmrg2d_autotune(ops.ptr, int(precision), C.byref(best), ms, N_TILE_CONFIGS,
                                 _stream(stream)))
    return best.value, list(ms)


def set_tile_config(ops: Ops, precision, index: int):
    precision = PRECISION.get(precision, precision)
    _check(lib().dmrg2d_set_tile_config(ops.ptr, int(precision), int(index)))


def tile_config_name(index: int) -> str:
    return lib().dmrg2d_tile_config_name(int(index)).decode()


def default_solver_opts() -> dict:
    o = SolverOpts()
    lib().dmrg2d_default_solver_opts(C.byref(o))
    return {k: getattr(o, k) for k, _ in SolverOpts._fields_}


def lanczos_ground(ops: Ops, x, stream=None, **opts):
    """Ground state; x (CUDA float64, n_vec) is the start vector and receives the result.

    Returns (energy, stats dict, status code).  ENOCONV is returned, not raised.
    """
    o = default_solver_opts()
    for k, v in opts.items():
        if k not in o:
            raise KeyError(k)
        o[k] = PRECISION.get(v, v) if k in ("precision", "refine_precision") else v
    so = SolverOpts(**o)
    if not x.is_cuda or str(x.dtype) != "torch.float64" or x.numel() != ops.info["n_vec"]:
        raise ValueError("x must be a CUDA float64 tensor of n_vec elements")
    e = C.c_double()
    st = SolverStats()
    code = lib().dmrg2d_lanczos_ground(ops.ptr, C.byref(so), C.c_void_p(x.data_ptr()), C.byref(e),
                                       C.byref(st), _stream(stream))
    if code not in (0, -5):
        _check(code)
    return e.value, {k: getattr(st, k) for k, _ in SolverStats._fields_}, code


def lanczos_ground_noalloc(ops: Ops, x, stream=None, **opts):
    """dmrg2d_lanczos_ground_noalloc: the plain FP64 solve of lanczos_ground with all of
    its scratch in the library's static device array, so the call allocates nothing.

    For callers that cannot call cudaMalloc (device memory owned by another allocator,
    or loops that cannot take cudaMalloc's implicit synchronisation).  Small
    superblocks only: (krylov_dim + 2) * n_vec plus small arrays must fit in
    DMRG2D_NOALLOC_SCRATCH_DOUBLES doubles.  Returns (energy, stats, status).
    """
    o = default_solver_opts()
    for k, v in opts.items():
        if k not in o:
            raise KeyError(k)
        o[k] = PRECISION.get(v, v) if k in ("precision", "refine_precision") else v
    so = SolverOpts(**o)
    if not x.is_cuda or str(x.dtype) != "torch.float64" or x.numel() != ops.info["n_vec"]:
        raise ValueError("x must be a CUDA float64 tensor of n_vec elements")
    e = C.c_double()
    st = SolverStats()
    code = lib().dmrg2d_lanczos_ground_noalloc(ops.ptr, C.byref(so), C.c_void_p(x.data_ptr()),
                                               C.byref(e), C.byref(st), _stream(stream))
    if code not in (0, -5):
        _check(code)
    return e.value, {k: getattr(st, k) for k, _ in SolverStats._fields_}, code


def tridiag_lowest(alpha, beta, stream=None):
    """Lowest eigenpair of the tridiagonal (alpha, beta[:k-1]) on the device
    (dmrg2d_tridiag_lowest); alpha, beta: CUDA float64 tensors of k elements.
    Returns (eigenvalue, eigenvector tensor, residual estimate |beta[k-1] s[k-1]|, status)."""
    import torch
    k = alpha.numel()
    for t in (alpha, beta):
        if not t.is_cuda or str(t.dtype) != "torch.float64" or t.numel() != k:
            raise ValueError("alpha, beta: CUDA float64 tensors of equal length")
    s = torch.empty(k, dtype=torch.float64, device=alpha.device)
    out = torch.empty(3 + 5 * k, dtype=torch.float64, device=alpha.device)
    _check(lib().dmrg2d_tridiag_lowest(C.c_void_p(alpha.data_ptr()), C.c_void_p(beta.data_ptr()),
                                       int(k), C.c_void_p(s.data_ptr()),
                                       C.c_void_p(out.data_ptr()), _stream(stream)))
    o = out[:3].cpu().numpy()
    return float(o[0]), s, float(o[1]), int(o[2])


PRECOND = {"none": 0, "jacobi": 1, "mlp": 2}
SWEEP_SOLVER = {"lanczos": 0, "davidson": 1}


def site_densities(ops: Ops, x, stream=None) -> dict:
    """Densities of the two central columns' sites for the state x (CUDA float64, n_vec):
    n[c, y, s] (c = 0 column 2, 1 column 3; s = 0 up, 1 down), hole density h[c, y],
    staggered spin density sd[c, y] and S[c] = max_y |sd[c, y]| (dmrg2d_site_densities)."""
    import torch
    if not x.is_cuda or str(x.dtype) != "torch.float64" or x.numel() != ops.info["n_vec"]:
        raise ValueError("x must be a CUDA float64 tensor of n_vec elements")
    nl = ops.info["n_legs"]
    out = torch.empty(8 * nl + 2, dtype=torch.float64, device=x.device)
    _check(lib().dmrg2d_site_densities(ops.ptr, C.c_void_p(x.data_ptr()),
                                       C.c_void_p(out.data_ptr()), _stream(stream)))
    o = out.cpu().numpy()
    per = o[:8 * nl].reshape(2, nl, 4)
    return {"n": per[..., :2].copy(), "h": per[..., 2].copy(), "sd": per[..., 3].copy(),
            "S": o[8 * nl:].copy()}


def diagonal(ops: Ops, out, stream=None):
    """out (CUDA float64, n_vec) = diagonal of H in the vector layout."""
    if not out.is_cuda or str(out.dtype) != "torch.float64" or out.numel() != ops.info["n_vec"]:
        raise ValueError("out must be a CUDA float64 tensor of n_vec elements")
    _check(lib().dmrg2d_diagonal(ops.ptr, C.c_void_p(out.data_ptr()), _stream(stream)))


def davidson_ground(ops: Ops, x, stream=None, mlp=None, log=None, **opts):
    """Davidson; x (CUDA float64) is the start vector and receives the result.

    log: optional (cap, x_log, r_log) with CUDA float64 tensors of cap*n_vec elements;
    returns (energy, stats, status[, thetas]).
    """
    o = DavidsonOpts()
    lib().dmrg2d_default_davidson_opts(C.byref(o))
    for k, v in opts.items():
        if k == "precision":
            v = PRECISION.get(v, v)
        if k == "precond":
            v = PRECOND.get(v, v)
        setattr(o, k, v)
    if mlp is not None:
        o.mlp = mlp.ptr
    thetas = None
    if log is not None:
        cap, xl, rl = log
        thetas = (C.c_double * cap)()
        o.log_cap = cap
        o.log_x = xl.data_ptr() if xl is not None else None
        o.log_r = rl.data_ptr() if rl is not None else None
        o.log_theta = thetas
    if not x.is_cuda or str(x.dtype) != "torch.float64" or x.numel() != ops.info["n_vec"]:
        raise ValueError("x must be a CUDA float64 tensor of n_vec elements")
    e = C.c_double()
    st = SolverStats()
    code = lib().dmrg2d_davidson_ground(ops.ptr, C.byref(o), C.c_void_p(x.data_ptr()), C.byref(e),
                                        C.byref(st), _stream(stream))
    if code not in (0, -5):
        _check(code)
    stats = {k: getattr(st, k) for k, _ in SolverStats._fields_}
    if thetas is not None:
        return e.value, stats, code, list(thetas)
    return e.value, stats, code


class MLP:
    """The learned preconditioner's network (device parameters, FP32)."""

    def __init__(self, hidden=256, seed=0):
        p = C.c_void_p()
        _check(lib().dmrg2d_mlp_create(int(hidden), int(seed), C.byref(p)))
        self._p = p
        self.hidden = hidden
        self.n_params = lib().dmrg2d_mlp_num_params(p)

    @property
    def ptr(self):
        return self._p

    def free(self):
        if self._p:
            lib().dmrg2d_mlp_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        h = np.empty(self.n_params, dtype=np.float32)
        _check(lib().dmrg2d_mlp_get_params(self._p, h.ctypes.data_as(C.c_void_p)))
        return h

    def set_params(self, h):
        h = np.ascontiguousarray(h, dtype=np.float32)
        assert h.size == self.n_params
        _check(lib().dmrg2d_mlp_set_params(self._p, h.ctypes.data_as(C.c_void_p)))

    def forward(self, X, Y, stream=None):
        _check(lib().dmrg2d_mlp_forward(self._p, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                        int(Y.numel()), _stream(stream)))

    def loss_grad(self, X, w, T, grad, stream=None):
        loss = C.c_float()
        _check(lib().dmrg2d_mlp_loss_grad(self._p, C.c_void_p(X.data_ptr()), C.c_void_p(w.data_ptr()),
                                          C.c_void_p(T.data_ptr()), int(T.numel()),
                                          C.c_void_p(grad.data_ptr()), C.byref(loss),
                                          _stream(stream)))
        return loss.value

    def train_step(self, X, w, T, lr, stream=None):
        loss = C.c_float()
        _check(lib().dmrg2d_mlp_train_step(self._p, C.c_void_p(X.data_ptr()), C.c_void_p(w.data_ptr()),
                                           C.c_void_p(T.data_ptr()), int(T.numel()), float(lr),
                                           C.byref(loss), _stream(stream)))
        return loss.value


def mlp_make_batch(ops: Ops, x_k, r_k, theta, x_final, D, idx, X, w, T, stream=None):
    _check(lib().dmrg2d_mlp_make_batch(
        ops.ptr, C.c_void_p(x_k.data_ptr()), C.c_void_p(r_k.data_ptr()), float(theta),
        C.c_void_p(x_final.data_ptr()), C.c_void_p(D.data_ptr()), C.c_void_p(idx.data_ptr()),
        int(idx.numel()), C.c_void_p(X.data_ptr()), C.c_void_p(w.data_ptr()),
        C.c_void_p(T.data_ptr()), _stream(stream)))


class SweepState:
    """A DMRG run that continues across calls (dmrg2d_state): the warm-up on the first
    sweep() call, then the requested sweeps on every call, each starting where the last
    one stopped.  model, n_columns, m_warmup, seed, sectors, n_up, n_dn are fixed here;
    the solver options may change per call."""

    def __init__(self, model: dict, n_columns: int, m_warmup: int, seed=1, sectors=False,
                 n_up=0, n_dn=0):
        self.model = model
        self._fixed = dict(n_columns=int(n_columns), m_warmup=int(m_warmup), seed=int(seed),
                           use_sectors=int(bool(sectors)), n_up=int(n_up), n_dn=int(n_dn))
        opts = self._opts([], FP64, 1e-10, 300, 100, {})
        mdl = _model(model)
        p = C.c_void_p()
        _check(lib().dmrg2d_state_create(C.byref(mdl), C.byref(opts[0]), C.byref(p)))
        self._p = p

    def _opts(self, m_sweeps, precision, tol, max_iter, krylov_dim, dav):
        ms = (C.c_int * max(1, len(m_sweeps)))(*[int(m) for m in m_sweeps])
        f = self._fixed
        mlp = dav.get("mlp")
        o = SweepOpts(f["n_columns"], f["m_warmup"], len(m_sweeps), ms, int(precision),
                      float(tol), int(max_iter), int(krylov_dim), f["seed"], f["use_sectors"],
                      f["n_up"], f["n_dn"], SWEEP_SOLVER[dav.get("solver", "lanczos")],
                      PRECOND.get(dav.get("precond", "jacobi"), dav.get("precond")),
                      mlp.ptr if mlp is not None else None, int(dav.get("mlp_train_sweeps", 1)),
                      int(dav.get("mlp_epochs", 1)))
        return o, ms

    def sweep(self, m_sweeps, precision=FP64, tol=1e-10, max_iter=300, krylov_dim=100,
              cap=4096, stream=None, solver="lanczos", precond="jacobi", mlp=None,
              mlp_train_sweeps=1, mlp_epochs=1) -> dict:
        """One finite sweep per entry of m_sweeps (after the warm-up on the first call);
        the per-step report as dmrg2d.sweep returns it.  solver "davidson" takes the
        Davidson solver with precond "none" / "jacobi" / "mlp"; with "mlp" the network
        `mlp` is trained in place on the warm-up's solves and those of the sweeps with
        index < mlp_train_sweeps (mlp_epochs passes; 0: used as given)."""
        precision = PRECISION.get(precision, precision)
        opts, ms = self._opts(m_sweeps, precision, tol, max_iter, krylov_dim,
                              dict(solver=solver, precond=precond, mlp=mlp,
                                   mlp_train_sweeps=mlp_train_sweeps, mlp_epochs=mlp_epochs))
        e, t = (C.c_double * cap)(), (C.c_double * cap)()
        ll, sw, it = (C.c_int * cap)(), (C.c_int * cap)(), (C.c_int * cap)()
        nl = int(self.model["n_legs"])
        nr = max(nl - 1, 1)
        leg, rung, s2 = (C.c_double * (cap * nl))(), (C.c_double * (cap * nr))(), (C.c_double * cap)()
        nd = 8 * nl + 2
        dens = (C.c_double * (cap * nd))()
        rep = SweepReport(cap, 0, e, t, ll, sw, it, leg, rung, s2, dens, 0.0, 0.0, 0.0, 0.0, 0.0,
                          0.0, 0.0, 0.0)
        _check(lib().dmrg2d_sweep(self._p, C.byref(opts), C.byref(rep), _stream(stream)))
        n = min(rep.n_steps, cap)
        return {"energy": list(e[:n]), "trunc": list(t[:n]), "l": list(ll[:n]),
                "sweep": list(sw[:n]), "iters": list(it[:n]),
                "leg_bond": [list(leg[i * nl:(i + 1) * nl]) for i in range(n)],
                "rung_bond": [list(rung[i * nr:(i + 1) * nr])[:nl - 1] for i in range(n)],
                "s2": list(s2[:n]), "obs_seconds": rep.obs_seconds,
                "n_steps": rep.n_steps, "seconds": rep.seconds,
                "solve_seconds": rep.solve_seconds, "build_seconds": rep.build_seconds,
                "dm_seconds": rep.dm_seconds, "renorm_seconds": rep.renorm_seconds,
                "train_seconds": rep.train_seconds, "transform_seconds": rep.transform_seconds,
                **_sweep_densities(dens, n, nl)}

    def info(self) -> dict:
        inf = StateInfo()
        _check(lib().dmrg2d_state_get_info(self._p, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in StateInfo._fields_}

    def free(self):
        if self._p:
            lib().dmrg2d_state_free(self._p)
            self._p = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sweep(model: dict, n_columns: int, m_warmup: int, m_sweeps, precision=FP64, tol=1e-10,
          max_iter=300, krylov_dim=100, seed=1, cap=4096, sectors=False, n_up=0, n_dn=0,
          stream=None, **davidson) -> dict:
    """dmrg2d_sweep on a fresh state: warm-up plus one finite sweep per entry of m_sweeps
    on an n-leg Heisenberg ladder (or, with sectors=True and the filling n_up, n_dn, a
    Hubbard ladder) of n_columns columns.  Returns the per-step energy, truncation error,
    block-1 length and sweep index (-1 = warm-up), the observables and the timings; for
    Hubbard ladders "n" (steps x 2 columns x n_legs x [up, down]), "h", "sd" (steps x 2 x
    n_legs) and "S" (steps x 2) are the central columns' site densities.  The keyword
    arguments solver, precond, mlp, mlp_train_sweeps, mlp_epochs are SweepState.sweep's."""
    st = SweepState(model, n_columns, m_warmup, seed=seed, sectors=sectors, n_up=n_up,
                    n_dn=n_dn)
    try:
        return st.sweep(m_sweeps, precision=precision, tol=tol, max_iter=max_iter,
                        krylov_dim=krylov_dim, cap=cap, stream=stream, **davidson)
    finally:
        st.free()


def _sweep_densities(buf, n: int, nl: int) -> dict:
    """Split the report's per-step density records (layout of dmrg2d_site_densities)."""
    a = np.frombuffer(buf, dtype=np.float64, count=n * (8 * nl + 2)).reshape(n, 8 * nl + 2)
    per = a[:, :8 * nl].reshape(n, 2, nl, 4)
    return {"n": per[..., :2].copy(), "h": per[..., 2].copy(), "sd": per[..., 3].copy(),
            "S": a[:, 8 * nl:].copy()}
