"""Host-side checks of the C-ABI library: it loads, exports every symbol its
header declares, and its host-only size query agrees with the oracle's mesh."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_11520_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2008_11520_gb300 import dnnmg
    return dnnmg


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|size_t|const char \*)\s*(dnnmg_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for n in ("dnnmg_prolongate", "dnnmg_patch_features", "dnnmg_gru_step", "dnnmg_scatter_avg",
              "dnnmg_rhs_restrict", "dnnmg_step", "dnnmg_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(so, n)]
    assert not missing


@pytest.mark.parametrize("cfg", [
    dict(nxc=32, nyc=8, K=1, s=1, ellipse=(0.2, 0.2, 0.04, 0.06)),
    dict(nxc=64, nyc=16, K=2, s=2, ellipse=(0.2, 0.2, 0.05, 0.04)),
    dict(nxc=38, nyc=10, K=1, s=2, ellipse=(0.3, 0.2, 0.1, 0.08)),
    dict(nxc=16, nyc=8, K=3, s=1, ellipse=None),
])
def test_mesh_query_matches_oracle(lib, cfg):
    from oracle.mesh import Mesh
    om = Mesh(cfg["nxc"], cfg["nyc"], cfg["K"], cfg["s"], ellipse=cfg["ellipse"])
    info = lib.dnnmg_mesh_query(lib.make_desc(cfg["nxc"], cfg["nyc"], cfg["K"], cfg["s"], cfg["ellipse"]))
    assert (info.P, info.nf, info.nc, info.n_in, info.n_out) == (om.P, om.nf, om.nc, om.n_in, om.n_out)
    assert (info.Nf, info.Nc) == (om.Nf, om.Nc)
    assert info.n_solid_coarse == int(om.solid_coarse.sum())
    assert info.ldx % 16 == 0 and info.ldx >= info.n_in


def test_mesh_query_explicit_mask(lib):
    from oracle.mesh import Mesh
    rng = np.random.default_rng(0)
    mask = rng.random((8, 16)) < 0.3
    om = Mesh(16, 8, 1, 2, solid=mask)
    info = lib.dnnmg_mesh_query(lib.make_desc(16, 8, 1, 2, solid=mask))
    assert info.P == om.P and info.n_solid_coarse == int(mask.sum())


@pytest.mark.parametrize("bad", [dict(nxc=31), dict(K=0), dict(K=4), dict(s=3), dict(nxc=30, s=4),
                                 dict(precision=7)])
def test_mesh_query_rejects_invalid(lib, bad):
    args = dict(nxc=32, nyc=8, K=1, s=1)
    prec = bad.pop("precision", "f64")
    args.update(bad)
    with pytest.raises(lib.DnnmgError) as e:
        lib.dnnmg_mesh_query(lib.make_desc(args["nxc"], args["nyc"], args["K"], args["s"], precision=prec))
    assert e.value.code in (1, 3) and str(e.value)


def test_mesh_query_rejects_oversize(lib):
    with pytest.raises(lib.DnnmgError) as e:
        lib.dnnmg_mesh_query(lib.make_desc(1024, 16384, 2, 1))
    assert e.value.code == 3


def _run_isolated(code, pythonpath):
    import subprocess
    import sys
    env = dict(os.environ, PYTHONPATH=pythonpath)
    return subprocess.run([sys.executable, "-c", code], cwd=pythonpath, env=env,
                          capture_output=True, text=True, timeout=300)


def test_product_modules_never_load_the_oracle(lib):
    # the oracle is test infrastructure: no module of the package may import it
    mods = ["dnnmg", "synth", "solver", "timeloop", "train", "serve", "build"]
    code = ("import sys\n"
            + "".join(f"import paper_2008_11520_gb300.{m}\n" for m in mods)
            + "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            + "assert not bad, bad\n")
    r = _run_isolated(code, ROOT)
    assert r.returncode == 0, r.stderr[-2000:]


def test_binding_fails_loudly_without_the_library(tmp_path):
    # a copy of the package without libdnnmg.so: importing the binding raises
    # ImportError (no fallback), while host-only modules still import
    import shutil
    src = os.path.join(ROOT, "paper_2008_11520_gb300")
    dst = tmp_path / "paper_2008_11520_gb300"
    dst.mkdir()
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), dst / f)
    code = ("import paper_2008_11520_gb300.solver\n"
            "try:\n"
            "    import paper_2008_11520_gb300.dnnmg\n"
            "except ImportError as e:\n"
            "    assert 'libdnnmg.so is missing' in str(e) and 'no fallback' in str(e), e\n"
            "else:\n"
            "    raise SystemExit('imported without the library')\n")
    r = _run_isolated(code, str(tmp_path))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def test_plain_c_client_links_and_queries(lib, tmp_path):
    # The boundary is a C ABI: a C99 program that includes only the header
    # compiles, takes the address of every declared entry point (so each links
    # from libdnnmg.so), and runs the host-only size query and head-size query
    # without a GPU, agreeing with the binding.
    import shutil
    import subprocess
    from paper_2008_11520_gb300 import build, synth
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    syms = sorted(declared_symbols())
    c = synth.config("large")
    cx, cy, ax, ay = c["ellipse"]
    src = "\n".join([
        "#include <stdio.h>",
        '#include "dnnmg.h"',
        "static void *const entry_points[] = {" + ", ".join(f"(void *)&{s}" for s in syms) + "};",
        "int main(void) {",
        "    dnnmg_mesh_desc d = {0};",
        "    dnnmg_mesh_info info;",
        f"    d.nxc = {c['nxc']}; d.nyc = {c['nyc']}; d.K = {c['K']}; d.s = {c['s']};",
        f"    d.lx = 2.2; d.ly = 0.41; d.obst_cx = {cx!r}; d.obst_cy = {cy!r}; d.obst_ax = {ax!r}; d.obst_ay = {ay!r};",
        "    d.nu = 1e-3; d.k = 0.01; d.alpha0 = 0.1; d.u_max = 1.5; d.precision = DNNMG_F32;",
        "    if (dnnmg_mesh_query(&d, &info) != DNNMG_OK) { printf(\"error %s\\n\", dnnmg_last_error()); return 1; }",
        "    printf(\"%d %lld %lld %d %d %d %d\\n\", info.P, info.Nf, info.Nc, info.n_in, info.n_out, info.ldx,",
        "           dnnmg_head_params(18));",
        "    d.K = 7;",
        "    if (dnnmg_mesh_query(&d, &info) != DNNMG_EINVAL) return 2;",
        "    return entry_points[0] == 0;",
        "}",
    ])
    (tmp_path / "client.c").write_text(src)
    exe = str(tmp_path / "client")
    libdir = os.path.dirname(build.LIB)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                        str(tmp_path / "client.c"), "-o", exe, "-L", libdir, "-ldnnmg", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    P, Nf, Nc, n_in, n_out, ldx, nt = (int(v) for v in r.stdout.split())
    info = lib.dnnmg_mesh_query(lib.make_desc(c["nxc"], c["nyc"], c["K"], c["s"], c["ellipse"], precision="f32"))
    assert (P, Nf, Nc, n_in, n_out, ldx) == (info.P, info.Nf, info.Nc, info.n_in, info.n_out, info.ldx)
    assert nt == 90
