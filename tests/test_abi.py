"""C-ABI library: builds, loads and exports every declared symbol; host-side validation (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0707_0159_gb300 import build, dmrg2d
    if not os.path.exists(build.LIB):
        build.build()
    return dmrg2d.lib()


def declared_symbols():
    syms = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(dmrg2d_\w+)\s*\(", txt))
    return sorted(syms)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "dmrg2d_apply_H" in syms and "dmrg2d_build_ops" in syms
    so = ctypes.CDLL(os.path.join(ROOT, "paper_0707_0159_gb300", "libdmrg2d.so"))
    for s in syms:
        assert hasattr(so, s), s


def test_binding_covers_header(lib):
    from paper_0707_0159_gb300 import dmrg2d
    assert set(declared_symbols()) == set(dmrg2d.SIGNATURES)


def test_version_and_error_text(lib):
    from paper_0707_0159_gb300 import dmrg2d
    assert "sm_103a" in dmrg2d.version()
    assert isinstance(dmrg2d.last_error(), str)


def test_build_ops_rejects_bad_input_on_host(lib):
    """Argument checks run before any device call, so they work without a GPU."""
    from paper_0707_0159_gb300 import dmrg2d, synth
    mdl = synth.model("heisenberg", 2)
    good = synth.heisenberg_block(4, 2, 0)
    bad = dict(good)
    bad["edge"] = good["edge"][:3]           # n_edge must be 0 or 2*n_legs
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.build_ops(mdl, bad, good)
    assert e.value.code == -2 and "n_edge" in str(e.value)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.build_ops(dict(mdl, n_legs=0), good, good)
    assert e.value.code == -1
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.build_ops(dict(mdl, n_legs=11), good, good)
    assert e.value.code == -1


def test_default_solver_opts(lib):
    from paper_0707_0159_gb300 import dmrg2d
    o = dmrg2d.default_solver_opts()
    assert o["precision"] == dmrg2d.FP64 and o["max_iter"] > 0 and o["tol"] > 0


def test_wait_selftest_rejects_bad_limits(lib):
    from paper_0707_0159_gb300 import dmrg2d
    assert dmrg2d.wait_selftest(0.0) == -1      # EINVAL before any device work
    assert dmrg2d.wait_selftest(5.0) == -1


def test_sweep_rejects_bad_options(lib):
    from paper_0707_0159_gb300 import dmrg2d, synth
    mdl = synth.model("heisenberg", 2, J_leg=1.0, J_rung=1.0)
    for kw in (dict(n_columns=5), dict(n_columns=2), dict(m_warmup=0), dict(tol=0.0)):
        args = dict(n_columns=6, m_warmup=8, m_sweeps=[8], tol=1e-10)
        args.update(kw)
        n_columns, m_warmup = args.pop("n_columns"), args.pop("m_warmup")
        with pytest.raises(dmrg2d.Dmrg2dError) as e:
            dmrg2d.sweep(mdl, n_columns, m_warmup, **args)
        assert e.value.code == -1
    hub = synth.model("hubbard", 2, t=1.0, U=8.0)
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.sweep(hub, 6, 8, [8])
    assert e.value.code == -8


def test_site_densities_rejects_null_arguments(lib):
    import ctypes
    assert lib.dmrg2d_site_densities(None, None, None, None) == -1      # EINVAL, no device work
    assert "NULL" in lib.dmrg2d_last_error().decode()
    buf = (ctypes.c_double * 4)()
    assert lib.dmrg2d_site_densities(None, buf, buf, None) == -1


def test_sweep_state_is_created_and_validated_on_host(lib):
    """dmrg2d_state_create checks the lattice and filling before any device work."""
    from paper_0707_0159_gb300 import dmrg2d, synth
    st = dmrg2d.SweepState(synth.model("heisenberg", 2), 6, 16)
    info = st.info()
    assert info["n_columns"] == 6 and info["warmed_up"] == 0 and info["sweeps_done"] == 0
    assert info["failed"] == 0
    st.free()
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.SweepState(synth.model("heisenberg", 2), 5, 16)        # odd lattice
    assert e.value.code == -1
    with pytest.raises(dmrg2d.Dmrg2dError) as e:                       # Hubbard needs sectors
        dmrg2d.SweepState(synth.model("hubbard", 2), 6, 16, sectors=False)
    assert e.value.code == -8
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        dmrg2d.SweepState(synth.model("hubbard", 2), 6, 16, sectors=True, n_up=13)
    assert e.value.code == -1


@pytest.mark.parametrize("kw", [dict(solver="davidson", precond=7),
                                dict(solver="davidson", precond="mlp", mlp=None),
                                dict(solver="davidson", precond="mlp", mlp_epochs=-1)])
def test_sweep_solver_options_are_validated_on_host(lib, kw):
    """The sweep's solver fields (unknown preconditioner, the learned one without a
    network, negative epochs) are refused before the first device call."""
    from paper_0707_0159_gb300 import dmrg2d, synth
    st = dmrg2d.SweepState(synth.model("heisenberg", 2), 6, 8)
    if kw.get("mlp_epochs") == -1:
        class _Net:                      # any non-NULL pointer passes the NULL check
            ptr = 1
        kw = dict(kw, mlp=_Net())
    with pytest.raises(dmrg2d.Dmrg2dError) as e:
        st.sweep([8], **kw)
    assert e.value.code == -1
    assert st.info()["failed"] == 0 and st.info()["warmed_up"] == 0
    st.free()


def test_sweep_rejects_an_unknown_solver(lib):
    from paper_0707_0159_gb300 import dmrg2d, synth
    st = dmrg2d.SweepState(synth.model("heisenberg", 2), 6, 8)
    opts, ms = st._opts([8], dmrg2d.FP64, 1e-10, 300, 100, {})
    opts.solver = 5
    rep = dmrg2d.SweepReport()
    rep.cap = 0
    assert dmrg2d.lib().dmrg2d_sweep(st._p, dmrg2d.C.byref(opts), dmrg2d.C.byref(rep), None) == -1
    assert st.info()["failed"] == 0
    st.free()


def test_mirrored_structs_match_the_library(lib):
    """Every struct the binding mirrors has the size the library was compiled with (a
    field added on one side only would shift every later field)."""
    from paper_0707_0159_gb300 import dmrg2d
    C = dmrg2d.C
    pairs = [(0, dmrg2d.Model), (1, dmrg2d.Block), (2, dmrg2d.OpsInfo), (3, dmrg2d.SolverOpts),
             (4, dmrg2d.SolverStats), (5, dmrg2d.DavidsonOpts), (6, dmrg2d.SweepOpts),
             (7, dmrg2d.SweepReport), (8, dmrg2d.StateInfo)]
    for which, cls in pairs:
        assert dmrg2d.lib().dmrg2d_struct_size(which) == C.sizeof(cls), cls.__name__
    assert dmrg2d.lib().dmrg2d_struct_size(99) == 0


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """The boundary is a C ABI: include/dmrg2d.h compiles as C99 with warnings as errors,
    and a C program that calls the library through it links against libdmrg2d.so and
    runs (host-only calls: version, defaults, struct sizes)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text(
        '#include "dmrg2d.h"\n'
        "#include <stdio.h>\n"
        "int main(void) {\n"
        "  dmrg2d_solver_opts o;\n"
        "  dmrg2d_default_solver_opts(&o);\n"
        "  if (o.max_iter < 1) return 2;\n"
        "  if (dmrg2d_struct_size(DMRG2D_STRUCT_SWEEP_OPTS) != sizeof(dmrg2d_sweep_opts))\n"
        "    return 3;\n"
        "  if (dmrg2d_struct_size(DMRG2D_STRUCT_SWEEP_REPORT) != sizeof(dmrg2d_sweep_report))\n"
        "    return 4;\n"
        '  printf("%s\\n", dmrg2d_version());\n'
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "use"
    libdir = os.path.join(root, "paper_0707_0159_gb300")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-ldmrg2d",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "dmrg2d" in r.stdout
