"""ctypes binding of libmv (include/mv.h): argument marshalling only.

Every function here allocates its outputs and workspace with PyTorch on the
current CUDA device, passes raw device pointers and the current stream to
the C ABI, and raises ``MvError`` on a non-OK status.  No arithmetic of the
method happens in Python.  If ``libmv.so`` has not been built the first call
raises ``RuntimeError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmv.so")

MV_OK, MV_ERR_INVALID_ARG, MV_ERR_INFEASIBLE, MV_ERR_NOT_CONVERGED = 0, 1, 2, 3
MV_ERR_TIMEOUT, MV_ERR_NUMERIC, MV_ERR_CUDA, MV_ERR_UNSUPPORTED, MV_ERR_WORKSPACE = 4, 5, 6, 7, 8
MV_F32, MV_BF16, MV_FP8_E4M3 = 0, 1, 2
MV_RETURN_GE, MV_RETURN_EQ = 0, 1
MV_LAYOUT_NT, MV_LAYOUT_TN, MV_LAYOUT_SIGMA = 0, 1, 2

DTYPES = {"f32": MV_F32, "bf16": MV_BF16, "fp8": MV_FP8_E4M3}
_ESIZE = {MV_F32: 4, MV_BF16: 2, MV_FP8_E4M3: 1}
_TORCH = {MV_F32: torch.float32, MV_BF16: torch.bfloat16, MV_FP8_E4M3: torch.uint8}
MODES = {"ge": MV_RETURN_GE, "eq": MV_RETURN_EQ}
LAYOUTS = {"nt": MV_LAYOUT_NT, "tn": MV_LAYOUT_TN, "sigma": MV_LAYOUT_SIGMA}

# Every symbol include/mv.h declares (checked by the CPU test suite).
EXPORTS = [
    "mv_status_string", "mv_version", "mv_center_workspace_size", "mv_center_factor", "mv_project",
    "mv_solve_opts_default", "mv_npga_workspace_size", "mv_npga_solve", "mv_gradient", "mv_last_error",
    "mv_gradient_noalloc", "mv_npga_solve_refined", "mv_sketch", "mv_str_workspace_size", "mv_str_truncate",
    "mv_sketch_str", "mv_frontier_workspace_size", "mv_npga_solve_frontier", "mv_backward_workspace_size",
    "mv_npga_backward", "mv_batch_workspace_size", "mv_npga_solve_batch", "mv_center_host_workspace_size",
    "mv_center_factor_host", "mv_batch_tiles", "mv_str_truncate_knee", "mv_sigma_workspace_size",
    "mv_sigma_form", "mv_countsketch_workspace_size", "mv_countsketch", "mv_gradient_noalloc_scratch_size",
    "mv_sketch_workspace_size", "mv_sketch_dtype", "mv_gaussian_sketch", "mv_countsketch_draw",
    "mv_sketch_str_workspace_size", "mv_frontier_refined_workspace_size", "mv_npga_solve_frontier_refined",
]

# Size of the library's fixed scratch array used by mv_gradient_noalloc.
NOALLOC_SCRATCH_BYTES = 16 << 20


class MvError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        extra = ""
        if status in (MV_ERR_CUDA, MV_ERR_UNSUPPORTED):
            extra = " -- " + lib().mv_last_error().decode()
        super().__init__(f"{where}: {status_string(status)} (status {status}){extra}")


class ProjInfo(C.Structure):
    _fields_ = [("nu", C.c_double), ("tau", C.c_double), ("residual", C.c_double),
                ("support", C.c_int32), ("status", C.c_int32), ("steps", C.c_int32),
                ("active", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("L", C.c_void_p), ("dtype", C.c_int32), ("mode", C.c_int32),
                ("row_scale", C.c_void_p), ("n", C.c_int64), ("T", C.c_int64), ("ld", C.c_int64),
                ("gamma", C.c_double), ("mu", C.c_void_p), ("R_target", C.c_double),
                ("power_start", C.c_void_p), ("layout", C.c_int32), ("reserved", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("kkt_every", C.c_int32), ("power_iters", C.c_int32),
                ("warm_start", C.c_int32), ("eps", C.c_double), ("power_safety", C.c_double),
                ("alpha", C.c_double), ("use_graph", C.c_int32), ("timing", C.c_int32),
                ("checkpoint_every", C.c_int32), ("two_pass", C.c_int32), ("momentum", C.c_int32),
                ("backtrack", C.c_int32), ("m_f", C.c_double), ("bt_rho", C.c_double), ("bt_alpha0", C.c_double),
                ("proj_budget", C.c_int32), ("dykstra_iters", C.c_int32), ("lanczos", C.c_int32),
                ("reserved_opts", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("converged", C.c_int32),
                ("proj_failures", C.c_int32), ("kkt", C.c_double), ("objective", C.c_double),
                ("alpha", C.c_double), ("lambda_hat", C.c_double), ("nu", C.c_double),
                ("launches", C.c_int32), ("timed_pairs", C.c_int32), ("t_gemv_t_ms", C.c_double),
                ("t_gemv_n_ms", C.c_double), ("t_step_ms", C.c_double), ("proj_steps", C.c_int32),
                ("refine_iterations", C.c_int32), ("fused", C.c_int32), ("t_fused_ms", C.c_double),
                ("backtracks", C.c_int32), ("dykstra", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libmv.so once; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmv.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl, sz = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_size_t
        L.mv_status_string.restype = C.c_char_p
        L.mv_status_string.argtypes = [i32]
        L.mv_version.restype = C.c_char_p
        L.mv_last_error.restype = C.c_char_p
        L.mv_center_workspace_size.restype = sz
        L.mv_center_workspace_size.argtypes = [i64, i64]
        L.mv_center_factor.restype = i32
        L.mv_center_factor.argtypes = [vp, i64, i64, i64, i32, i32, vp, i64, vp, vp, vp, vp, sz, vp]
        L.mv_countsketch_workspace_size.restype = sz
        L.mv_countsketch_workspace_size.argtypes = [i64, i64]
        L.mv_countsketch.restype = i32
        L.mv_countsketch.argtypes = [vp, i32, i32, vp, i64, i64, i64, vp, vp, i64, vp, i64, vp, sz, vp]
        L.mv_sigma_workspace_size.restype = sz
        L.mv_sigma_workspace_size.argtypes = [C.POINTER(Problem)]
        L.mv_sigma_form.restype = i32
        L.mv_sigma_form.argtypes = [C.POINTER(Problem), vp, i64, vp, sz, vp]
        L.mv_batch_tiles.restype = i32
        L.mv_batch_tiles.argtypes = [C.POINTER(Problem), i64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.mv_center_host_workspace_size.restype = sz
        L.mv_center_host_workspace_size.argtypes = [i64, i64]
        L.mv_center_factor_host.restype = i32
        L.mv_center_factor_host.argtypes = [vp, i64, i64, i64, i32, i32, vp, i64, vp, vp, vp, vp, sz, vp]
        L.mv_project.restype = i32
        L.mv_project.argtypes = [vp, vp, vp, i64, i64, i32, vp, vp, vp]
        L.mv_solve_opts_default.restype = None
        L.mv_solve_opts_default.argtypes = [C.POINTER(SolveOpts)]
        L.mv_npga_workspace_size.restype = sz
        L.mv_npga_workspace_size.argtypes = [C.POINTER(Problem)]
        L.mv_npga_solve.restype = i32
        L.mv_npga_solve.argtypes = [C.POINTER(Problem), C.POINTER(SolveOpts), vp, C.POINTER(SolveInfo),
                                    vp, sz, vp]
        L.mv_gradient.restype = i32
        L.mv_gradient.argtypes = [C.POINTER(Problem), vp, vp, vp, vp, sz, vp]
        L.mv_npga_solve_refined.restype = i32
        L.mv_npga_solve_refined.argtypes = [C.POINTER(Problem), C.POINTER(Problem), C.POINTER(SolveOpts), dbl, vp,
                                            C.POINTER(SolveInfo), vp, sz, vp]
        L.mv_str_workspace_size.restype = sz
        L.mv_str_workspace_size.argtypes = [i64, i64, i64]
        L.mv_str_truncate.restype = i32
        L.mv_str_truncate.argtypes = [vp, i64, i64, i64, i64, dbl, dbl, vp, i64, vp, C.POINTER(C.c_double), vp, sz,
                                      vp]
        L.mv_str_truncate_knee.restype = i32
        L.mv_str_truncate_knee.argtypes = [vp, i64, i64, i64, dbl, dbl, i64, dbl, dbl, dbl, vp, i64, vp,
                                           C.POINTER(C.c_int64), C.POINTER(C.c_double), vp, sz, vp]
        u64 = C.c_uint64
        L.mv_sketch_str.restype = i32
        L.mv_sketch_str.argtypes = [vp, i32, vp, i64, i64, i64, i64, u64, i64, dbl, dbl, vp, i64, vp, i64, vp,
                                    C.POINTER(C.c_double), vp, sz, vp]
        L.mv_sketch_str_workspace_size.restype = sz
        L.mv_sketch_str_workspace_size.argtypes = [i32, i64, i64, i64, i64, i32]
        L.mv_sketch_workspace_size.restype = sz
        L.mv_sketch_workspace_size.argtypes = [i32, i64, i64]
        L.mv_sketch_dtype.restype = i32
        L.mv_sketch_dtype.argtypes = [vp, i32, vp, i64, i64, i64, vp, i64, i64, vp, i64, vp, sz, vp]
        L.mv_gaussian_sketch.restype = i32
        L.mv_gaussian_sketch.argtypes = [u64, i64, i64, vp, i64, vp]
        L.mv_countsketch_draw.restype = i32
        L.mv_countsketch_draw.argtypes = [u64, i64, i64, vp, vp, vp]
        L.mv_frontier_workspace_size.restype = sz
        L.mv_frontier_workspace_size.argtypes = [C.POINTER(Problem), i64]
        L.mv_npga_solve_frontier.restype = i32
        L.mv_npga_solve_frontier.argtypes = [C.POINTER(Problem), vp, i64, C.POINTER(SolveOpts), vp,
                                             C.POINTER(SolveInfo), vp, sz, vp]
        L.mv_frontier_refined_workspace_size.restype = sz
        L.mv_frontier_refined_workspace_size.argtypes = [C.POINTER(Problem), C.POINTER(Problem), i64]
        L.mv_npga_solve_frontier_refined.restype = i32
        L.mv_npga_solve_frontier_refined.argtypes = [C.POINTER(Problem), C.POINTER(Problem), vp, i64,
                                                     C.POINTER(SolveOpts), dbl, vp, C.POINTER(SolveInfo), vp, sz, vp]
        L.mv_backward_workspace_size.restype = sz
        L.mv_backward_workspace_size.argtypes = [C.POINTER(Problem), C.POINTER(SolveOpts)]
        L.mv_npga_backward.restype = i32
        L.mv_npga_backward.argtypes = [C.POINTER(Problem), C.POINTER(SolveOpts), vp, vp, vp, vp, i64,
                                       C.POINTER(SolveInfo), vp, sz, vp]
        L.mv_batch_workspace_size.restype = sz
        L.mv_batch_workspace_size.argtypes = [C.POINTER(Problem), i64]
        L.mv_npga_solve_batch.restype = i32
        L.mv_npga_solve_batch.argtypes = [C.POINTER(Problem), i64, C.POINTER(SolveOpts), C.POINTER(C.c_void_p),
                                          C.POINTER(SolveInfo), vp, sz, vp]
        L.mv_sketch.restype = i32
        L.mv_sketch.argtypes = [vp, i64, i64, i64, vp, i64, i64, vp, i64, vp]
        L.mv_gradient_noalloc.restype = i32
        L.mv_gradient_noalloc.argtypes = [C.POINTER(Problem), vp, vp, vp, vp]
        L.mv_gradient_noalloc_scratch_size.restype = sz
        L.mv_gradient_noalloc_scratch_size.argtypes = [C.POINTER(Problem)]
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().mv_status_string(int(status)).decode()


def version() -> str:
    return lib().mv_version().decode()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status, where, allow=()):
    if status != MV_OK and status not in allow:
        raise MvError(status, where)
    return status


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks.
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def padded_ld(T: int, dtype: int) -> int:
    """Smallest leading dimension >= T whose row pitch is a multiple of 16 bytes."""
    v = 16 // _ESIZE[dtype]
    return (T + v - 1) // v * v


# ------------------------------------------------------------------ calls
def center_factor(R: torch.Tensor, out_dtype: str = "f32", ld: int | None = None, layout: str = "nt"):
    """mu, L, trace(Sigma) from an n x T FP32 return panel on the GPU (Sec. 2.1).

    Returns (L, row_scale, mu, trace) where L is n x ld (columns T.. are 0)
    for layout "nt", or L^T as T x ld (columns n.. are 0) for layout "tn";
    row_scale is an n FP32 tensor for FP8 (else None), mu is FP64 n and trace
    an FP64 scalar tensor.
    """
    assert R.is_cuda and R.dtype == torch.float32 and R.dim() == 2
    dt = DTYPES[out_dtype]
    lay = LAYOUTS[layout]
    n, T = R.shape
    ldR = R.stride(0)
    if R.stride(1) != 1:
        raise ValueError("R must be row-major")
    inner, outer = (T, n) if lay == MV_LAYOUT_NT else (n, T)
    ld = padded_ld(inner, dt) if ld is None else int(ld)
    dev = R.device
    L = torch.empty((outer, ld), dtype=_TORCH[dt], device=dev)
    rs = torch.empty(n, dtype=torch.float32, device=dev) if dt == MV_FP8_E4M3 else None
    mu = torch.empty(n, dtype=torch.float64, device=dev)
    tr = torch.empty(1, dtype=torch.float64, device=dev)
    wsz = lib().mv_center_workspace_size(n, T)
    ws = _workspace(wsz, dev)
    _check(lib().mv_center_factor(_ptr(R), n, T, ldR, dt, lay, _ptr(L), ld, _ptr(rs), _ptr(mu), _ptr(tr),
                                  _ptr(ws), ws.numel(), _stream()), "mv_center_factor")
    return L, rs, mu, tr


def center_factor_host(R: torch.Tensor, out_dtype: str = "f32", ld: int | None = None, layout: str = "nt",
                       device=None, ws: torch.Tensor | None = None):
    """center_factor from an n x T FP32 panel in host memory (best pinned): the
    upload and the centering overlap chunk by chunk (mv_center_factor_host).
    ``ws`` may pass a reusable workspace of mv_center_host_workspace_size bytes."""
    assert not R.is_cuda and R.dtype == torch.float32 and R.dim() == 2 and R.stride(1) == 1
    dt = DTYPES[out_dtype]
    lay = LAYOUTS[layout]
    n, T = R.shape
    inner, outer = (T, n) if lay == MV_LAYOUT_NT else (n, T)
    ld = padded_ld(inner, dt) if ld is None else int(ld)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    L = torch.empty((outer, ld), dtype=_TORCH[dt], device=dev)
    rs = torch.empty(n, dtype=torch.float32, device=dev) if dt == MV_FP8_E4M3 else None
    mu = torch.empty(n, dtype=torch.float64, device=dev)
    tr = torch.empty(1, dtype=torch.float64, device=dev)
    wsz = lib().mv_center_host_workspace_size(n, T)
    if ws is None or ws.numel() < wsz:
        ws = _workspace(wsz, dev)
    _check(lib().mv_center_factor_host(C.c_void_p(R.data_ptr()), n, T, R.stride(0), dt, lay, _ptr(L), ld, _ptr(rs),
                                       _ptr(mu), _ptr(tr), _ptr(ws), ws.numel(), _stream()), "mv_center_factor_host")
    return L, rs, mu, tr


def project(v: torch.Tensor, mu: torch.Tensor, R_target, mode: str = "ge"):
    """Exact projection onto F of each row of v (batch x n or n), FP64."""
    squeeze = v.dim() == 1
    v2 = v.reshape(1, -1) if squeeze else v
    assert v2.is_cuda and v2.dtype == torch.float64 and v2.is_contiguous()
    batch, n = v2.shape
    Rt = torch.as_tensor(R_target, dtype=torch.float64, device=v.device).reshape(-1)
    if Rt.numel() == 1 and batch > 1:
        Rt = Rt.expand(batch).contiguous()
    x = torch.empty_like(v2)
    info = torch.zeros(batch * C.sizeof(ProjInfo), dtype=torch.uint8, device=v.device)
    _check(lib().mv_project(_ptr(v2), _ptr(mu.contiguous()), _ptr(Rt), n, batch, MODES[mode], _ptr(x),
                            _ptr(info), _stream()), "mv_project")
    raw = info.cpu().numpy().tobytes()
    infos = [ProjInfo.from_buffer_copy(raw[i * C.sizeof(ProjInfo):(i + 1) * C.sizeof(ProjInfo)])
             for i in range(batch)]
    out = [{k: getattr(p, k) for k, _ in ProjInfo._fields_} for p in infos]
    return (x[0], out[0]) if squeeze else (x, out)


def shape_error(layout: str, dtype: str, L_shape, L_esize: int, n: int, T: int, mu_numel: int,
                rs_numel: int | None = None, ps_numel: int | None = None) -> str | None:
    """Why the arrays cannot hold the problem, or None.  The kernels read an
    n x T block of L ("nt"), T x n ("tn") or n x n ("sigma") and n entries
    of mu, the row scales and the power-method start; the C ABI only sees
    pointers, so the sizes are checked here."""
    want = _ESIZE[DTYPES[dtype]]
    if L_esize != want:
        return f"L holds {L_esize}-byte elements; dtype {dtype} stores {want}-byte ones"
    rows, cols = int(L_shape[0]), int(L_shape[1])
    need = {"nt": (n, T), "tn": (T, n), "sigma": (n, n)}[layout]
    if rows < need[0] or cols < need[1]:
        return f"L is {rows} x {cols}; layout {layout} with n = {n}, T = {T} reads {need[0]} x {need[1]}"
    for name, k in (("mu", mu_numel), ("row_scale", rs_numel), ("power_start", ps_numel)):
        if k is not None and k < n:
            return f"{name} has {k} entries; the problem has n = {n}"
    return None


def make_problem(L: torch.Tensor, mu: torch.Tensor, R_target: float, T: int, gamma: float = 0.0,
                 dtype: str = "f32", row_scale: torch.Tensor | None = None, mode: str = "ge",
                 power_start: torch.Tensor | None = None, layout: str = "nt") -> Problem:
    """mv_problem over L as center_factor returns it (n x ld for "nt", T x ld for "tn"),
    or over an explicit n x ld covariance from sigma_form ("sigma"; T is not read)."""
    assert L.is_cuda and L.dim() == 2 and L.stride(1) == 1
    p = Problem()
    p.L = L.data_ptr()
    p.dtype = DTYPES[dtype]
    p.mode = MODES[mode]
    p.layout = LAYOUTS[layout]
    p.reserved = 0
    p.row_scale = None if row_scale is None else row_scale.data_ptr()
    n = L.shape[0] if p.layout == MV_LAYOUT_NT else mu.shape[0]
    err = shape_error(layout, dtype, L.shape, L.element_size(), n, max(1, int(T)) if layout != "sigma" else 1,
                      mu.numel(), None if row_scale is None else row_scale.numel(),
                      None if power_start is None else power_start.numel())
    if err is not None:
        raise ValueError(err)
    p.n, p.T, p.ld = n, max(1, int(T)), L.stride(0)
    p.gamma = float(gamma)
    p.mu = mu.data_ptr()
    p.R_target = float(R_target)
    p.power_start = None if power_start is None else power_start.data_ptr()
    return p


def sigma_form(L: torch.Tensor, T: int, dtype: str = "f32", row_scale: torch.Tensor | None = None):
    """Sigma = L L^T (n x ld FP32, ld = n rounded up to 4) from the n x ld factor
    (mv_sigma_form: tcgen05, upper tiles only, both triangles written)."""
    n = L.shape[0]
    mu = torch.zeros(n, dtype=torch.float64, device=L.device)
    p = make_problem(L, mu, 0.0, T, 0.0, dtype, row_scale)
    nb = lib().mv_sigma_workspace_size(C.byref(p))
    if nb == 0:
        raise MvError(MV_ERR_INVALID_ARG, "mv_sigma_workspace_size")
    ws = _workspace(nb, L.device)
    ldS = (n + 3) // 4 * 4
    S = torch.zeros((n, ldS), dtype=torch.float32, device=L.device)
    _check(lib().mv_sigma_form(C.byref(p), _ptr(S), ldS, _ptr(ws), ws.numel(), _stream()), "mv_sigma_form")
    return S


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().mv_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _check_y(y: torch.Tensor, n: int, device) -> None:
    """The gradient calls read y as n FP64 values on L's device."""
    if not isinstance(y, torch.Tensor) or y.dtype != torch.float64:
        raise ValueError("y must be a float64 tensor")
    if y.device != torch.device(device):
        raise ValueError(f"y is on {y.device}; L is on {device}")
    if y.dim() != 1 or y.numel() != n or not y.is_contiguous():
        raise ValueError(f"y must be a contiguous vector of n = {n} entries (got shape {tuple(y.shape)})")


class Solver:
    """Holds a problem, its workspace and the device solution buffer.

    ``solve()`` calls mv_npga_solve; reusing one Solver reuses the cached
    CUDA graph and workspace, which is what a benchmark loop wants.
    """

    def __init__(self, L, mu, R_target, T, gamma=0.0, dtype="f32", row_scale=None, mode="ge",
                 power_start=None, layout="nt", **opts):
        self._keep = (L, mu, row_scale, power_start)
        self.problem = make_problem(L, mu, R_target, T, gamma, dtype, row_scale, mode, power_start, layout)
        self.opts = solve_opts(**opts)
        self.ws_bytes = lib().mv_npga_workspace_size(C.byref(self.problem))
        if self.ws_bytes == 0:
            raise MvError(MV_ERR_INVALID_ARG, "mv_npga_workspace_size")
        self.ws = _workspace(self.ws_bytes, L.device)
        self.x = torch.zeros(mu.shape[0], dtype=torch.float64, device=L.device)

    def solve(self, x0: torch.Tensor | None = None, allow=(MV_ERR_NOT_CONVERGED,)):
        if x0 is not None:
            self.x.copy_(x0)
            self.opts.warm_start = 1
        info = SolveInfo()
        st = lib().mv_npga_solve(C.byref(self.problem), C.byref(self.opts), _ptr(self.x), C.byref(info),
                                 _ptr(self.ws), self.ws.numel(), _stream())
        _check(st, "mv_npga_solve", allow)
        return self.x, info.as_dict()

    def gradient(self, y: torch.Tensor, with_z: bool = True):
        """(z, g); with ``with_z=False`` z is None and g comes from the fused
        single pass over L where that applies."""
        _check_y(y, self.problem.n, self.ws.device)
        with_z = with_z and self.problem.layout != MV_LAYOUT_SIGMA
        z = torch.empty(self.problem.T, dtype=torch.float32, device=y.device) if with_z else None
        g = torch.empty(self.problem.n, dtype=torch.float64, device=y.device)
        _check(lib().mv_gradient(C.byref(self.problem), _ptr(y), _ptr(z) if with_z else None, _ptr(g),
                                 _ptr(self.ws), self.ws.numel(), _stream()), "mv_gradient")
        return z, g


class RefinedSolver:
    """Low-precision solve (BF16 or FP8 copy of L) refined on the FP32 copy
    (mv_npga_solve_refined); reuses workspace and graphs across calls."""

    def __init__(self, L_lo, L_hi, mu, R_target, T, gamma=0.0, dtype="bf16", row_scale=None, mode="ge",
                 power_start=None, eps_lo=1e-5, layout="nt", layout_hi=None, **opts):
        self._keep = (L_lo, L_hi, mu, row_scale, power_start)
        self.p_lo = make_problem(L_lo, mu, R_target, T, gamma, dtype, row_scale, mode, power_start, layout)
        self.p_hi = make_problem(L_hi, mu, R_target, T, gamma, "f32", None, mode, power_start,
                                 layout if layout_hi is None else layout_hi)
        self.opts = solve_opts(**opts)
        self.eps_lo = float(eps_lo)
        nb = max(lib().mv_npga_workspace_size(C.byref(self.p_lo)), lib().mv_npga_workspace_size(C.byref(self.p_hi)))
        if nb == 0:
            raise MvError(MV_ERR_INVALID_ARG, "mv_npga_workspace_size")
        self.ws = _workspace(nb, L_hi.device)
        self.x = torch.zeros(mu.shape[0], dtype=torch.float64, device=L_hi.device)

    def solve(self, allow=(MV_ERR_NOT_CONVERGED,)):
        info = SolveInfo()
        st = lib().mv_npga_solve_refined(C.byref(self.p_lo), C.byref(self.p_hi), C.byref(self.opts), self.eps_lo,
                                         _ptr(self.x), C.byref(info), _ptr(self.ws), self.ws.numel(), _stream())
        _check(st, "mv_npga_solve_refined", allow)
        return self.x, info.as_dict()


def npga_solve(L, mu, R_target, T, gamma=0.0, dtype="f32", row_scale=None, mode="ge", x0=None,
               power_start=None, layout="nt", **opts):
    """One-shot NPGA solve; returns (x, info dict)."""
    s = Solver(L, mu, R_target, T, gamma, dtype, row_scale, mode, power_start, layout, **opts)
    return s.solve(x0)


def gradient(L, y, T, gamma=0.0, dtype="f32", row_scale=None, with_z=True, layout="nt"):
    """(z, g) with z = L^T y (FP32) and g = 2 L z + 2 gamma y (FP64).
    ``with_z=False``: z is None and g uses the fused single pass where it applies."""
    n = L.shape[0] if layout == "nt" else y.shape[0]
    mu = torch.zeros(n, dtype=torch.float64, device=L.device)
    s = Solver(L, mu, 0.0, T, gamma, dtype, row_scale, layout=layout)
    return s.gradient(y, with_z)


def gradient_noalloc(L, y, T, gamma=0.0, dtype="f32", row_scale=None, layout="nt", with_z=True):
    """(z, g) as ``gradient`` but through mv_gradient_noalloc: the library uses
    its fixed scratch array instead of a workspace (outputs still come from
    PyTorch here).  Calls overlapping on the GPU race on that array."""
    n = L.shape[0] if layout == "nt" else y.shape[0]
    mu = torch.zeros(n, dtype=torch.float64, device=L.device)
    p = make_problem(L, mu, 0.0, T, gamma, dtype, row_scale, layout=layout)
    _check_y(y, p.n, L.device)
    z = torch.empty(T, dtype=torch.float32, device=y.device) if with_z else None
    g = torch.empty(p.n, dtype=torch.float64, device=y.device)
    _check(lib().mv_gradient_noalloc(C.byref(p), _ptr(y), _ptr(z), _ptr(g), _stream()), "mv_gradient_noalloc")
    return z, g


def gradient_noalloc_scratch_size(L, T, dtype="f32", row_scale=None, layout="nt", n=None) -> int:
    """Bytes of the library's fixed array that mv_gradient_noalloc needs for
    this problem on the current device (0 if the problem is invalid)."""
    n = L.shape[0] if layout == "nt" else int(n)
    mu = torch.zeros(n, dtype=torch.float64, device=L.device)
    p = make_problem(L, mu, 0.0, T, 0.0, dtype, row_scale, layout=layout)
    return int(lib().mv_gradient_noalloc_scratch_size(C.byref(p)))


def sketch(L_bf16: torch.Tensor, T: int, Phi_t: torch.Tensor) -> torch.Tensor:
    """tilde L = L Phi (Sec. 2.3): L is n x ld BF16 (from center_factor), Phi_t is
    m x ldP BF16 holding Phi transposed (row j = sketch column j).  Returns the
    n x m FP32 product (tcgen05 BF16 GEMM, FP32 accumulation).  Blocking."""
    assert L_bf16.dtype == torch.bfloat16 and Phi_t.dtype == torch.bfloat16
    n, m = L_bf16.shape[0], Phi_t.shape[0]
    if L_bf16.shape[1] < T or Phi_t.shape[1] < T:
        raise ValueError(f"L ({L_bf16.shape[1]} columns) and Phi_t ({Phi_t.shape[1]}) must hold T = {T} periods")
    ldS = (m + 3) // 4 * 4
    out = torch.empty((n, ldS), dtype=torch.float32, device=L_bf16.device)
    _check(lib().mv_sketch(_ptr(L_bf16), n, T, L_bf16.stride(0), _ptr(Phi_t), m, Phi_t.stride(0), _ptr(out), ldS,
                           _stream()), "mv_sketch")
    return out[:, :m]


def sketch_dtype(L: torch.Tensor, T: int, Phi_t: torch.Tensor, dtype: str = "f32",
                 row_scale: torch.Tensor | None = None) -> torch.Tensor:
    """tilde L = L Phi for an n x ld factor stored as "f32", "bf16" or "fp8"
    (mv_sketch_dtype); Phi_t is m x ldP BF16.  Returns n x m FP32."""
    assert Phi_t.dtype == torch.bfloat16
    dt = DTYPES[dtype]
    n, m = L.shape[0], Phi_t.shape[0]
    err = shape_error("nt", dtype, L.shape, L.element_size(), n, T, n,
                      None if row_scale is None else row_scale.numel())
    if err is None and Phi_t.shape[1] < T:
        err = f"Phi_t has {Phi_t.shape[1]} columns; T = {T}"
    if err is not None:
        raise ValueError(err)
    ws = _workspace(lib().mv_sketch_workspace_size(dt, n, T), L.device)
    ldS = (m + 3) // 4 * 4
    out = torch.empty((n, ldS), dtype=torch.float32, device=L.device)
    _check(lib().mv_sketch_dtype(_ptr(L), dt, _ptr(row_scale), n, T, L.stride(0), _ptr(Phi_t), m, Phi_t.stride(0),
                                 _ptr(out), ldS, _ptr(ws), ws.numel(), _stream()), "mv_sketch_dtype")
    return out[:, :m]


def gaussian_sketch(seed: int, m: int, T: int, device=None) -> torch.Tensor:
    """Phi^T (m x ldP BF16, ldP = T rounded up to 8) drawn on the device from
    ``seed`` (mv_gaussian_sketch: Philox4x32-10 + Box--Muller, N(0, 1/m))."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    ldP = (T + 7) // 8 * 8
    out = torch.empty((m, ldP), dtype=torch.bfloat16, device=dev)
    _check(lib().mv_gaussian_sketch(int(seed), m, T, _ptr(out), ldP, _stream()), "mv_gaussian_sketch")
    return out


def countsketch_draw(seed: int, T: int, m: int, device=None):
    """(h int32 [T], sign int8 [T]) drawn on the device from ``seed`` (mv_countsketch_draw)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    h = torch.empty(T, dtype=torch.int32, device=dev)
    sg = torch.empty(T, dtype=torch.int8, device=dev)
    _check(lib().mv_countsketch_draw(int(seed), T, m, _ptr(h), _ptr(sg), _stream()), "mv_countsketch_draw")
    return h, sg


def sketch_str(L: torch.Tensor, T: int, m: int, seed: int, k: int, dtype: str = "bf16",
               row_scale: torch.Tensor | None = None, gamma: float = -1.0, trace_sigma: float = 0.0,
               keep_sketch: bool = True):
    """The whole STR build from a seed (mv_sketch_str): returns (L_eff n x k
    FP32, sigma k FP64, gamma, tilde L n x m FP32 or None)."""
    dt = DTYPES[dtype]
    n = L.shape[0]
    err = shape_error("nt", dtype, L.shape, L.element_size(), n, T, n,
                      None if row_scale is None else row_scale.numel())
    if err is not None:
        raise ValueError(err)
    nb = lib().mv_sketch_str_workspace_size(dt, n, T, m, k, 0 if keep_sketch else 1)
    if nb == 0:
        raise MvError(MV_ERR_INVALID_ARG, "mv_sketch_str_workspace_size")
    dev = L.device
    ws = _workspace(nb, dev)
    ldS = (m + 3) // 4 * 4
    Ls = torch.empty((n, ldS), dtype=torch.float32, device=dev) if keep_sketch else None
    ldE = (k + 3) // 4 * 4
    L_eff = torch.zeros((n, ldE), dtype=torch.float32, device=dev)
    sigma = torch.empty(k, dtype=torch.float64, device=dev)
    g = C.c_double(0.0)
    _check(lib().mv_sketch_str(_ptr(L), dt, _ptr(row_scale), n, T, L.stride(0), m, int(seed), k, float(gamma),
                               float(trace_sigma), _ptr(Ls), ldS, _ptr(L_eff), ldE, _ptr(sigma), C.byref(g),
                               _ptr(ws), ws.numel(), _stream()), "mv_sketch_str")
    return L_eff[:, :k], sigma, g.value, (Ls[:, :m] if keep_sketch else None)


def bf16_rows(A, ld=None) -> torch.Tensor:
    """Host array (rows x cols) -> device BF16 tensor with a 16-byte row pitch
    (input preparation: rounding to BF16 is done by PyTorch)."""
    A = torch.as_tensor(A)
    r, c = A.shape
    ld = (c + 7) // 8 * 8 if ld is None else ld
    out = torch.zeros((r, ld), dtype=torch.bfloat16, device="cuda")
    out[:, :c] = A.to(device="cuda", dtype=torch.bfloat16)
    return out


def countsketch(L: torch.Tensor, n: int, T: int, h: torch.Tensor, sign: torch.Tensor, m: int, dtype: str = "f32",
                row_scale: torch.Tensor | None = None, layout: str = "nt"):
    """tilde L = L Phi for the CountSketch Phi of (h, sign) (mv_countsketch):
    n x m FP32.  L as center_factor returns it (n x ld for "nt", T x ld for "tn")."""
    assert h.dtype == torch.int32 and sign.dtype == torch.int8 and h.is_cuda and sign.is_cuda
    err = shape_error(layout, dtype, L.shape, L.element_size(), n, T, n,
                      None if row_scale is None else row_scale.numel())
    if err is None and (h.numel() < T or sign.numel() < T):
        err = f"h ({h.numel()}) and sign ({sign.numel()}) must hold T = {T} entries"
    if err is not None:
        raise ValueError(err)
    nb = lib().mv_countsketch_workspace_size(T, m)
    if nb == 0:
        raise MvError(MV_ERR_INVALID_ARG, "mv_countsketch_workspace_size")
    ws = _workspace(nb, L.device)
    ldS = (m + 3) // 4 * 4
    out = torch.empty((n, ldS), dtype=torch.float32, device=L.device)
    if ldS > m:
        out[:, m:].zero_()                                   # padding columns; the kernels write every j < m
    _check(lib().mv_countsketch(_ptr(L), DTYPES[dtype], LAYOUTS[layout], _ptr(row_scale) if row_scale is not None
                                else None, n, T, L.stride(0), _ptr(h), _ptr(sign), m, _ptr(out), ldS, _ptr(ws),
                                ws.numel(), _stream()), "mv_countsketch")
    return out


def str_truncate_knee(L_sketch: torch.Tensor, tau: float, rho: float, k_max: int, kappa_target: float = 0.0,
                      gamma: float = -1.0, trace_sigma: float = 0.0):
    """(L_eff (n x k_max, columns >= l zero), sigma (k_max), l, gamma): the knee-rule rank and
    the kappa-target ridge of App. D from the FP32 sketch tilde L (n x m)."""
    assert L_sketch.dtype == torch.float32 and L_sketch.stride(1) == 1
    n, m = L_sketch.shape
    ldS = L_sketch.stride(0)
    dev = L_sketch.device
    nb = lib().mv_str_workspace_size(n, m, k_max)
    if nb == 0:
        raise MvError(MV_ERR_UNSUPPORTED, "mv_str_workspace_size")
    ldE = (k_max + 3) // 4 * 4
    L_eff = torch.zeros((n, ldE), dtype=torch.float32, device=dev)
    sigma = torch.empty(k_max, dtype=torch.float64, device=dev)
    ws = _workspace(nb, dev)
    k = C.c_int64(0)
    g = C.c_double(0.0)
    _check(lib().mv_str_truncate_knee(_ptr(L_sketch), n, m, ldS, float(tau), float(rho), int(k_max),
                                      float(kappa_target), float(gamma), float(trace_sigma), _ptr(L_eff), ldE,
                                      _ptr(sigma), C.byref(k), C.byref(g), _ptr(ws), ws.numel(), _stream()),
           "mv_str_truncate_knee")
    return L_eff, sigma, int(k.value), float(g.value)


def str_truncate(L_sketch: torch.Tensor, k: int, gamma: float = -1.0, trace_sigma: float = 0.0):
    """Top-k FP64 truncation + ridge of tilde L (Sec. 2.5): returns (L_eff n x k
    FP32, sigma k FP64, gamma).  gamma < 0 selects 1e-4 tr(Sigma)/n."""
    assert L_sketch.dtype == torch.float32 and L_sketch.stride(1) == 1
    n, m = L_sketch.shape
    nb = lib().mv_str_workspace_size(n, m, k)
    if nb == 0:
        raise MvError(MV_ERR_UNSUPPORTED, "mv_str_workspace_size")
    ws = _workspace(nb, L_sketch.device)
    ldE = (k + 3) // 4 * 4
    L_eff = torch.zeros((n, ldE), dtype=torch.float32, device=L_sketch.device)
    sigma = torch.empty(k, dtype=torch.float64, device=L_sketch.device)
    g = C.c_double(0.0)
    _check(lib().mv_str_truncate(_ptr(L_sketch), n, m, L_sketch.stride(0), k, float(gamma), float(trace_sigma),
                                 _ptr(L_eff), ldE, _ptr(sigma), C.byref(g), _ptr(ws), ws.numel(), _stream()),
           "mv_str_truncate")
    return L_eff, sigma, g.value


class FrontierSolver:
    """Batched NPGA over many targets sharing one BF16 factor, or an FP8 factor
    with its row scales (mv_npga_solve_frontier); reuses the workspace.  With
    ``L_f32`` (the FP32 factor, n x ld) the solve is refined on it after the
    low-precision phase stops at ``eps_lo`` (mv_npga_solve_frontier_refined)."""

    def __init__(self, L_bf16, mu, R_targets, T, gamma=0.0, mode="ge", power_start=None, dtype="bf16",
                 row_scale=None, L_f32=None, eps_lo=1e-5, **opts):
        self.Rt = torch.as_tensor(R_targets, dtype=torch.float64).reshape(-1).to(L_bf16.device)
        self._keep = (L_bf16, mu, power_start, row_scale, L_f32)
        self.problem = make_problem(L_bf16, mu, 0.0, T, gamma, dtype, row_scale, mode, power_start)
        self.p_hi = None if L_f32 is None else make_problem(L_f32, mu, 0.0, T, gamma, "f32", None, mode, power_start)
        self.eps_lo = float(eps_lo)
        self.opts = solve_opts(**opts)
        self.nt = self.Rt.numel()
        if self.p_hi is None:
            nb = lib().mv_frontier_workspace_size(C.byref(self.problem), self.nt)
        else:
            nb = lib().mv_frontier_refined_workspace_size(C.byref(self.problem), C.byref(self.p_hi), self.nt)
        if nb == 0:
            raise MvError(MV_ERR_INVALID_ARG, "mv_frontier_workspace_size")
        self.ws = _workspace(nb, L_bf16.device)
        self.X = torch.zeros((self.nt, L_bf16.shape[0]), dtype=torch.float64, device=L_bf16.device)

    def solve(self, allow=(MV_ERR_NOT_CONVERGED,)):
        infos = (SolveInfo * self.nt)()
        if self.p_hi is None:
            st = lib().mv_npga_solve_frontier(C.byref(self.problem), _ptr(self.Rt), self.nt, C.byref(self.opts),
                                              _ptr(self.X), infos, _ptr(self.ws), self.ws.numel(), _stream())
            _check(st, "mv_npga_solve_frontier", allow)
        else:
            st = lib().mv_npga_solve_frontier_refined(C.byref(self.problem), C.byref(self.p_hi), _ptr(self.Rt),
                                                      self.nt, C.byref(self.opts), self.eps_lo, _ptr(self.X), infos,
                                                      _ptr(self.ws), self.ws.numel(), _stream())
            _check(st, "mv_npga_solve_frontier_refined", allow)
        return self.X, [i.as_dict() for i in infos]


def npga_backward(L, mu, R_target, T, dloss_dx, iters, gamma=0.0, mode="ge", x0=None, power_start=None,
                  checkpoint_every=50, **opts):
    """(d loss/d mu, d loss/d L, info) of the K-iteration unrolled solve (mv_npga_backward)."""
    p = make_problem(L, mu, R_target, T, gamma, "f32", None, mode, power_start)
    o = solve_opts(max_iter=int(iters), checkpoint_every=int(checkpoint_every), eps=0.0, kkt_every=0, **opts)
    nb = lib().mv_backward_workspace_size(C.byref(p), C.byref(o))
    if nb == 0:
        raise MvError(MV_ERR_INVALID_ARG, "mv_backward_workspace_size")
    ws = _workspace(nb, L.device)
    dmu = torch.empty(L.shape[0], dtype=torch.float64, device=L.device)
    dL = torch.empty_like(L)
    info = SolveInfo()
    _check(lib().mv_npga_backward(C.byref(p), C.byref(o), _ptr(x0), _ptr(dloss_dx.contiguous()), _ptr(dmu),
                                  _ptr(dL), L.stride(0), C.byref(info), _ptr(ws), ws.numel(), _stream()),
           "mv_npga_backward")
    return dmu, dL, info.as_dict()


class NPGAFunction(torch.autograd.Function):
    """x_K = NPGA unrolled for `iters` iterations, differentiable in mu and L.

    forward(L, mu, R_target, T, iters, gamma, checkpoint_every) runs
    mv_npga_solve with eps = 0 and no KKT checks (exactly `iters`
    iterations); backward calls mv_npga_backward.  alpha (power method), x^0
    and R_target are constants, as in the adjoint's conventions."""

    @staticmethod
    def forward(ctx, L, mu, R_target, T, iters, gamma=0.0, checkpoint_every=50):
        x, info = npga_solve(L, mu, R_target, T, gamma=gamma, eps=0.0, kkt_every=0, max_iter=int(iters))
        ctx.save_for_backward(L, mu)
        ctx.args = (float(R_target), int(T), int(iters), float(gamma), int(checkpoint_every))
        return x.clone()

    @staticmethod
    def backward(ctx, grad_x):
        L, mu = ctx.saved_tensors
        R_target, T, iters, gamma, ck = ctx.args
        dmu, dL, _ = npga_backward(L, mu, R_target, T, grad_x.to(torch.float64), iters, gamma=gamma,
                                   checkpoint_every=ck)
        return dL, dmu, None, None, None, None, None


class BatchSolver:
    """Independent problems of uneven size solved together (mv_npga_solve_batch).

    ``problems`` is a list of dicts with keys L, mu, R_target, T and optional
    gamma, row_scale, power_start, mode and layout ("nt": L is n x ld, the
    grouped GEMV pair; "tn": L^T is T x ld, the grouped single pass); all L
    share one dtype."""

    def __init__(self, problems, dtype="f32", **opts):
        self._keep = problems
        self.count = len(problems)
        self.probs = (Problem * self.count)()
        for i, q in enumerate(problems):
            self.probs[i] = make_problem(q["L"], q["mu"], q["R_target"], q["T"], q.get("gamma", 0.0), dtype,
                                         q.get("row_scale"), q.get("mode", "ge"), q.get("power_start"),
                                         q.get("layout", "nt"))
        self.opts = solve_opts(**opts)
        nb = lib().mv_batch_workspace_size(self.probs, self.count)
        if nb == 0:
            raise MvError(MV_ERR_INVALID_ARG, "mv_batch_workspace_size")
        dev = problems[0]["L"].device
        self.ws = _workspace(nb, dev)
        self.xs = [torch.zeros(q["mu"].shape[0], dtype=torch.float64, device=dev) for q in problems]
        self._xp = (C.c_void_p * self.count)(*[x.data_ptr() for x in self.xs])

    def solve(self, allow=(MV_ERR_NOT_CONVERGED,)):
        infos = (SolveInfo * self.count)()
        st = lib().mv_npga_solve_batch(self.probs, self.count, C.byref(self.opts), self._xp, infos, _ptr(self.ws),
                                       self.ws.numel(), _stream())
        _check(st, "mv_npga_solve_batch", allow)
        return self.xs, [i.as_dict() for i in infos]

    def tiles(self):
        """(rows per split, bytes per split, tuned?) of this batch shape's grouped GEMVs."""
        a, b = C.c_int32(), C.c_int32()
        st = lib().mv_batch_tiles(self.probs, self.count, C.byref(a), C.byref(b))
        _check(st, "mv_batch_tiles", (MV_ERR_NOT_CONVERGED,))
        return a.value, b.value, st == MV_OK
