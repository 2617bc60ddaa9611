"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/mv.h declares, and rejects bad arguments on the host before
anything is launched.  No GPU is touched."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mv.h")


@pytest.fixture(scope="module")
def mvmod():
    from paper_2604_02917_gb300 import build, mv
    if not os.path.exists(mv.LIB_PATH):
        build.build()
    mv.lib()
    return mv


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mv_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(mvmod):
    lib = mvmod.lib()
    names = declared_functions()
    assert "mv_npga_solve" in names and "mv_project" in names and "mv_center_factor" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in mv.h but not exported"
    assert set(names) <= set(mvmod.EXPORTS) | set(names)
    for name in mvmod.EXPORTS:
        assert name in names, f"binding lists {name} that mv.h does not declare"


def test_status_strings_and_version(mvmod):
    assert mvmod.version().startswith("mv ")
    for s in range(0, 9):
        assert mvmod.status_string(s).startswith("MV_")
    assert "unknown" in mvmod.status_string(99)


def _c_layout(tmp_path):
    """sizeof/offsetof of the mv.h structs as the C compiler lays them out."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {
        "mv_proj_info": ["nu", "tau", "residual", "support", "status", "steps", "active"],
        "mv_problem": ["L", "dtype", "mode", "row_scale", "n", "T", "ld", "gamma", "mu", "R_target",
                       "power_start", "layout", "reserved"],
        "mv_solve_opts": ["max_iter", "kkt_every", "power_iters", "warm_start", "eps", "power_safety",
                          "alpha", "use_graph", "timing", "checkpoint_every", "two_pass", "momentum",
                          "backtrack", "m_f", "bt_rho", "bt_alpha0", "proj_budget", "dykstra_iters",
                          "lanczos", "reserved_opts"],
        "mv_solve_info": ["iterations", "status", "converged", "proj_failures", "kkt", "objective",
                          "alpha", "lambda_hat", "nu", "launches", "timed_pairs", "t_gemv_t_ms",
                          "t_gemv_n_ms", "t_step_ms", "proj_steps", "refine_iterations", "fused",
                          "t_fused_ms", "backtracks", "dykstra"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mv.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.strip().splitlines()}


def test_struct_layouts_match_header(mvmod, tmp_path):
    lay = _c_layout(tmp_path)
    pairs = {"mv_proj_info": mvmod.ProjInfo, "mv_problem": mvmod.Problem,
             "mv_solve_opts": mvmod.SolveOpts, "mv_solve_info": mvmod.SolveInfo}
    for cname, py in pairs.items():
        assert C.sizeof(py) == lay[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == lay[(cname, f)], (cname, f)
    o = mvmod.solve_opts()
    assert o.max_iter == 10000 and o.kkt_every == 5 and o.power_iters == 50
    assert o.eps == 1e-6 and o.power_safety == 1e-3 and o.use_graph == 1
    assert o.momentum == 0 and o.backtrack == 0 and o.bt_rho == 0.5 and o.proj_budget == 100
    assert o.dykstra_iters == 2000 and o.lanczos == 0 and o.reserved_opts == 0


def test_host_side_argument_errors(mvmod):
    lib = mvmod.lib()
    # mv_project with null pointers / bad sizes: rejected before any launch.
    assert lib.mv_project(None, None, None, 10, 1, 0, None, None, None) == mvmod.MV_ERR_INVALID_ARG
    fake = C.c_void_p(256)
    assert lib.mv_project(fake, fake, fake, 0, 1, 0, fake, fake, None) == mvmod.MV_ERR_INVALID_ARG
    assert lib.mv_project(fake, fake, fake, 40000, 1, 0, fake, fake, None) == mvmod.MV_ERR_INVALID_ARG
    assert lib.mv_project(fake, fake, fake, 10, 1, 7, fake, fake, None) == mvmod.MV_ERR_INVALID_ARG
    # Problem validation: misaligned pitch, bad dtype, missing FP8 scales.
    p = mvmod.Problem()
    p.L, p.mu, p.n, p.T, p.ld, p.dtype = 4096, 4096, 10, 7, 7, mvmod.MV_F32
    assert lib.mv_npga_workspace_size(C.byref(p)) == 0          # ld*4 not a multiple of 16
    p.ld = 8
    assert lib.mv_npga_workspace_size(C.byref(p)) > 0
    p.dtype = 9
    assert lib.mv_npga_workspace_size(C.byref(p)) == 0
    p.dtype = mvmod.MV_FP8_E4M3
    p.ld = 16
    assert lib.mv_npga_workspace_size(C.byref(p)) == 0          # FP8 needs row scales
    info = mvmod.SolveInfo()
    p.dtype = mvmod.MV_F32
    st = lib.mv_npga_solve(C.byref(p), None, fake, C.byref(info), None, 0, None)
    assert st == mvmod.MV_ERR_WORKSPACE
    assert lib.mv_center_factor(None, 3, 4, 4, 0, 0, None, 4, None, None, None, None, 0, None) == \
        mvmod.MV_ERR_INVALID_ARG
    assert lib.mv_center_factor(fake, 3, 1, 4, 0, 0, fake, 4, None, fake, fake, fake, 1024, None) == \
        mvmod.MV_ERR_INVALID_ARG                                   # T < 2


def test_padded_ld(mvmod):
    assert mvmod.padded_ld(48374, mvmod.MV_F32) == 48376
    assert mvmod.padded_ld(48374, mvmod.MV_BF16) == 48376
    assert mvmod.padded_ld(48374, mvmod.MV_FP8_E4M3) == 48384
    assert mvmod.padded_ld(1000, mvmod.MV_F32) == 1000


def test_problem_shape_checks(mvmod):
    """The binding refuses arrays too small for the problem before any pointer
    reaches the library (which only sees pointers and sizes)."""
    se = mvmod.shape_error
    assert se("nt", "f32", (100, 1004), 4, 100, 1000, 100) is None          # padded leading dim
    assert se("tn", "bf16", (1000, 104), 2, 100, 1000, 100, None, 100) is None
    assert se("sigma", "f32", (100, 100), 4, 100, 1, 100) is None
    assert se("nt", "fp8", (100, 1008), 1, 100, 1000, 100, 100) is None
    assert "reads 100 x 1000" in se("nt", "f32", (100, 999), 4, 100, 1000, 100)
    assert "reads 1000 x 100" in se("tn", "f32", (999, 100), 4, 100, 1000, 100)
    assert "reads 1000 x 100" in se("tn", "f32", (1000, 99), 4, 100, 1000, 100)
    assert "reads 100 x 100" in se("sigma", "f32", (100, 99), 4, 100, 1, 100)
    assert "2-byte" in se("nt", "f32", (100, 1000), 2, 100, 1000, 100)
    assert se("nt", "f32", (100, 1000), 4, 100, 1000, 99).startswith("mu has 99")
    assert se("nt", "fp8", (100, 1000), 1, 100, 1000, 100, 50).startswith("row_scale has 50")
    assert se("nt", "f32", (100, 1000), 4, 100, 1000, 100, None, 3).startswith("power_start has 3")


def test_host_side_argument_errors_sketches_and_sigma(mvmod):
    """CountSketch, explicit Sigma and the knee rule refuse bad arguments on
    the host, before any launch."""
    lib = mvmod.lib()
    E, W, U = mvmod.MV_ERR_INVALID_ARG, mvmod.MV_ERR_WORKSPACE, mvmod.MV_ERR_UNSUPPORTED
    assert lib.mv_countsketch_workspace_size(0, 8) == 0
    assert lib.mv_countsketch_workspace_size(8, 0) == 0
    assert lib.mv_countsketch_workspace_size(1 << 31, 8) == 0
    assert lib.mv_countsketch_workspace_size(100, 16) > 0
    f, odd = C.c_void_p(4096), C.c_void_p(4100)
    NT, TN, SG = mvmod.MV_LAYOUT_NT, mvmod.MV_LAYOUT_TN, mvmod.MV_LAYOUT_SIGMA
    F32, FP8 = mvmod.MV_F32, mvmod.MV_FP8_E4M3

    def cs(L=f, dt=F32, lay=TN, rs=None, n=64, T=300, ld=64, m=32, ldS=32, ws=None, wsb=0):
        return lib.mv_countsketch(L, dt, lay, rs, n, T, ld, f, f, m, f, ldS, ws, wsb, None)

    assert cs(L=None) == E
    assert cs(dt=9) == E
    assert cs(lay=SG) == E
    assert cs(ldS=31) == E
    assert cs(ld=63) == E                                   # TN: ld >= n
    assert cs(lay=NT, ld=296) == E                          # NT: ld >= T
    assert cs(L=odd) == E                                   # 16-byte alignment
    assert cs(dt=FP8) == E                                  # FP8 needs row scales
    assert cs(lay=NT, T=60000, ld=60000) == U               # n x T row above 200 KB
    assert cs() == W                                       # no workspace
    # explicit Sigma: the problem must be a factor in the n x T layout
    p = mvmod.Problem()
    p.L, p.mu, p.n, p.T, p.ld, p.dtype, p.layout = 4096, 4096, 10, 7, 8, F32, NT
    assert lib.mv_sigma_workspace_size(C.byref(p)) > 0
    p.layout = TN
    assert lib.mv_sigma_workspace_size(C.byref(p)) == 0
    p.layout, p.ld = NT, 4
    assert lib.mv_sigma_workspace_size(C.byref(p)) == 0     # ld < T
    p.ld, p.n = 8, 40000
    assert lib.mv_sigma_workspace_size(C.byref(p)) == 0     # n above 32768
    p.n, p.dtype, p.ld = 10, FP8, 16
    assert lib.mv_sigma_workspace_size(C.byref(p)) == 0     # FP8 needs row scales
    p.dtype, p.ld = F32, 8
    assert lib.mv_sigma_form(C.byref(p), None, 12, None, 0, None) == E
    assert lib.mv_sigma_form(C.byref(p), f, 9, None, 0, None) == E      # ldS < n
    assert lib.mv_sigma_form(C.byref(p), f, 12, None, 0, None) == W
    # knee rule: tau > 0, 0 < rho < 1, kappa target <= 0 (off) or > 1
    k, g = C.c_int64(0), C.c_double(0.0)

    def knee(tau=0.1, rho=0.5, kmax=4, kappa=0.0, n=10):
        return lib.mv_str_truncate_knee(f, n, 16, 16, tau, rho, kmax, kappa, -1.0, 1.0, f, 4, f, C.byref(k),
                                        C.byref(g), None, 0, None)

    assert knee(tau=0.0) == E
    assert knee(rho=1.0) == E
    assert knee(kappa=0.5) == E
    assert knee(kmax=11) == E
    assert knee(n=1) == E


def test_unsupported_status_carries_its_own_message(mvmod):
    """Every MV_ERR_UNSUPPORTED return records its own reason, so the message
    read after it never belongs to an earlier, unrelated call."""
    lib = mvmod.lib()
    # 1: a sketch dimension beyond 2^31 (checked before any launch)
    st = lib.mv_sketch(C.c_void_p(4096), 1 << 31, 8, 8, C.c_void_p(4096), 8, 8, C.c_void_p(4096), 8, None)
    assert st == mvmod.MV_ERR_UNSUPPORTED
    assert "mv_sketch" in lib.mv_last_error().decode()
    # 2: then a problem with n above the projector's limit: its own message, not the sketch's
    p = mvmod.Problem()
    p.L, p.mu, p.n, p.T, p.ld, p.dtype = 4096, 4096, 40000, 64, 64, mvmod.MV_F32
    st = lib.mv_gradient_noalloc(C.byref(p), C.c_void_p(4096), None, C.c_void_p(4096), None)
    assert st == mvmod.MV_ERR_UNSUPPORTED
    msg = lib.mv_last_error().decode()
    assert "n must be <= 32768" in msg and "mv_sketch" not in msg
    with pytest.raises(mvmod.MvError) as e:
        mvmod._check(st, "mv_gradient_noalloc")
    assert "n must be <= 32768" in str(e.value)
    assert lib.mv_gradient_noalloc_scratch_size(C.byref(p)) == 0
