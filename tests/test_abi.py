"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every function include/cg.h declares, and rejects bad parameters on the host
(before any device call)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libcg():
    from paper_1407_5026_gb300 import build, binding
    build.build()
    return binding.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "cg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(cg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cg_create", "cg_run", "cg_read_state", "cg_observables",
                     "cg_write_state", "cg_destroy", "cg_create_batch", "cg_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libcg):
    for name in _declared():
        assert hasattr(libcg, name), name
    from paper_1407_5026_gb300 import binding
    assert sorted(binding.EXPORTED) == _declared()


def test_binding_structs_match_the_c_layout(libcg, tmp_path):
    # compile the header with the C compiler and compare sizes and offsets
    from paper_1407_5026_gb300 import binding as B
    structs = {"cg_replica_desc": B.cg_replica_desc, "cg_opts": B.cg_opts,
               "cg_counters": B.cg_counters, "cg_obs": B.cg_obs, "cg_hop": B.cg_hop}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cg.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        cname, field, val = line.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field)
    # the numpy record of cg_counters (batch state I/O) has the same layout
    dt = B.COUNTERS_DTYPE
    assert dt.itemsize == ctypes.sizeof(B.cg_counters)
    assert [(f, dt.fields[f][1]) for f in dt.names] == \
        [(f, getattr(B.cg_counters, f).offset) for f, _ in B.cg_counters._fields_]


@pytest.mark.parametrize("bad,msg", [
    (dict(L=15), "even"), (dict(L=2), "even"), (dict(nu=0.0), "nu"),
    (dict(L=6, nu=0.3), "integer"), (dict(r_max=8), "r_max"), (dict(xi=0.0), "xi"),
    (dict(T=0.0), "T must"), (dict(W=-1.0), "W must"), (dict(E=float("inf")), "E must"),
])
def test_create_rejects_bad_parameters_on_host(libcg, bad, msg):
    from paper_1407_5026_gb300 import binding as B
    p = dict(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=0)
    p.update(bad)
    with pytest.raises(B.CgError) as ei:
        B.cg_create(p["L"], p["nu"], p["W"], p["xi"], p["r_max"], p["T"], p["E"], p["seed"])
    assert msg in str(ei.value)


@pytest.mark.parametrize("bad,msg", [(dict(time_mode=2), "time_mode"),
                                     (dict(block_threads=300), "block_threads"),
                                     (dict(precision=7), "precision"),
                                     (dict(refresh_kind=7), "refresh_kind"),
                                     (dict(refresh_kind=-1), "refresh_kind"),
                                     (dict(pair_frac=1.0, pair_rmax=2), "pair_frac"),
                                     (dict(pair_frac=-0.1, pair_rmax=2), "pair_frac"),
                                     (dict(pair_frac=0.1, pair_rmax=0), "pair_rmax"),
                                     (dict(pair_frac=0.1, pair_rmax=8), "pair_rmax"),
                                     ])
def test_create_batch_rejects_bad_options_on_host(libcg, bad, msg):
    from paper_1407_5026_gb300 import binding as B
    with pytest.raises(B.CgError) as ei:
        B.cg_create_batch([B.desc(L=16)], B.opts(**bad))
    assert msg in str(ei.value)


def test_pair_offsets_must_fit_every_lattice_on_host(libcg):
    from paper_1407_5026_gb300 import binding as B
    with pytest.raises(B.CgError) as ei:
        B.cg_create_batch([B.desc(L=16), B.desc(L=6, r_max=2, dim=3)],
                          B.opts(pair_frac=0.2, pair_rmax=3))
    assert "pair_rmax" in str(ei.value)


def test_workspace_plan_counts_every_buffer(libcg):
    from paper_1407_5026_gb300 import binding as B
    reps = [B.desc(L=16), B.desc(L=16, seed=1), B.desc(L=32, r_max=6)]
    b64 = B.cg_workspace_bytes(reps, B.opts(precision=B.CG_FP64))
    b32 = B.cg_workspace_bytes(reps, B.opts(precision=B.CG_FP32,
                                            refresh_kind=B.CG_REFRESH_FP64))
    # eps shrinks by 4 bytes per site in binary32 (each buffer 256-aligned)
    assert b64 - b32 == 2 * 256 * 4 + 1024 * 4
    assert b64 % 256 == 0
    # the FFT refresh (L = 2^m or 3 2^m, the automatic choice) adds per group
    # a complex binary32 value per site and replica pair, DFT(g)/N (a
    # binary32 per site) and the L twiddles (8 bytes each), each 256-aligned
    fft = B.cg_workspace_bytes(reps, B.opts(precision=B.CG_FP32))
    up = lambda b: (b + 255) // 256 * 256
    extra = sum(up(((R + 1) // 2) * N * 8) + up(N * 4) + up(L * 8)
                for L, N, R in ((16, 256, 2), (32, 1024, 1)))
    assert fft - b32 == extra


def test_workspace_plan_counts_the_cubic_tensor_core_scratch(libcg):
    # 16 replicas of the 16^3 lattice in binary32: the tensor-core refresh adds
    # the +-1 image (2 N R_pad bytes), the K-split partials (k R_pad N x 4
    # bytes, k the smallest divisor of the N/64 K-blocks leaving at most 16 per
    # partial on the cubic lattice) and its 256-byte error word
    from paper_1407_5026_gb300 import binding as B
    reps = [B.desc(L=16, r_max=3, seed=s, replica=s, dim=3) for s in range(16)]
    tc = B.cg_workspace_bytes(reps, B.opts(precision=B.CG_FP32,
                                           refresh_kind=B.CG_REFRESH_BF16X2))
    plain = B.cg_workspace_bytes(reps, B.opts(precision=B.CG_FP32,
                                              refresh_kind=B.CG_REFRESH_FP64))
    N, R_pad, kblocks = 16 ** 3, 16, 16 ** 3 // 64
    k = next(d for d in range(1, kblocks + 1) if kblocks % d == 0 and kblocks // d <= 16)
    img = 2 * N * R_pad
    scratch = ((img + 255) // 256) * 256 + k * R_pad * N * 4
    assert tc - plain == ((scratch + 255) // 256) * 256 + 256


@pytest.mark.parametrize("L,R,nu,msg", [
    (15, 4, 0.5, "L must be even"), (1026, 4, 0.5, "L must be even"),
    (20, 4, 0.5, "multiple of 128"), (64, 0, 0.5, "R must be"), (64, 513, 0.5, "R must be"),
    (64, 4, 1.0, "nu must be"), (128, 49, 0.5, "static maximum"),
    (1024, 1, 0.5, "static maximum"),
])
def test_noalloc_refresh_refuses_bad_sizes_on_host(libcg, L, R, nu, msg):
    # every argument and size check comes before the first CUDA call, so the
    # refusals hold without a GPU; the buffers are host memory the refused
    # call never touches
    import numpy as np
    from paper_1407_5026_gb300 import binding as B
    buf = np.zeros(4, np.float64)
    with pytest.raises(B.CgError) as ei:
        B.cg_refresh_tc_noalloc(L, R, nu, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data)
    assert ei.value.code == B.CG_EINVAL
    assert msg in str(ei.value)
    with pytest.raises(B.CgError, match="required"):
        B.cg_refresh_tc_noalloc(64, 4, 0.5, 0, buf.ctypes.data, buf.ctypes.data)


def test_microbench_refuses_unknown_kinds_on_host(libcg):
    from paper_1407_5026_gb300 import binding as B
    for kind in (-1, 8):
        with pytest.raises(B.CgError, match="microbenchmark kind"):
            B.cg_microbench(kind, 0)


def test_missing_library_fails_loudly(tmp_path):
    # a fresh process whose library path points nowhere: every entry point
    # goes through load(), which raises instead of falling back to anything
    import subprocess
    import sys
    code = ("from paper_1407_5026_gb300 import binding as B\n"
            f"B.LIB_PATH = {str(tmp_path / 'libcg.so')!r}\n"
            "try:\n"
            "    B.cg_create(16, 0.5, 1.0, 1.0, 4, 0.05, 0.0, 0)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root,
                         timeout=120)
    assert "raised: libcg.so not built" in out.stdout, out.stdout + out.stderr


def test_product_package_has_no_cpu_path():
    # the package never imports the oracle, and no module of it computes the
    # chain in Python: the binding marshals arguments only
    import ast
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1407_5026_gb300")
    for name in os.listdir(pkg):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("oracle") for a in node.names), name
            if isinstance(node, ast.ImportFrom):
                assert not (node.module or "").startswith("oracle"), name


@pytest.mark.parametrize("bad,msg", [(dict(precision=1), "random sites"),
                                     (dict(pair_frac=0.1, pair_rmax=2), "random sites"),
                                     (dict(time_mode=1), "random sites")])
def test_random_sites_refuse_unsupported_options_on_host(libcg, bad, msg):
    from paper_1407_5026_gb300 import binding as B
    assert B.CG_FP32 == 1 and B.CG_TIME_GAUSSIAN == 1
    with pytest.raises(B.CgError) as ei:
        B.cg_create_batch([B.desc(L=16, sites=B.CG_SITES_RANDOM)], B.opts(**bad))
    assert msg in str(ei.value)


@pytest.mark.parametrize("kw,msg", [(dict(sites=2), "sites must"),
                                    (dict(sites=1, dim=3), "random sites")])
def test_random_site_descriptor_checks_on_host(libcg, kw, msg):
    from paper_1407_5026_gb300 import binding as B
    with pytest.raises(B.CgError) as ei:
        B.cg_create_batch([B.desc(L=16, **kw)], B.opts())
    assert msg in str(ei.value)


def test_random_sites_too_large_for_a_cluster_are_refused_at_once(libcg):
    # eps of a random-site replica lives in the shared memory of one CTA or
    # of a cluster of up to 8; L = 1024 (N = 2^20) is refused by the
    # descriptor check, before the site geometry would be built
    import time
    from paper_1407_5026_gb300 import binding as B
    big = [B.desc(L=1024, r_max=6, sites=B.CG_SITES_RANDOM)]
    t0 = time.perf_counter()
    with pytest.raises(B.CgError) as ei:
        B.cg_create_batch(big, B.opts())
    assert "L <= 362" in str(ei.value)
    assert B.cg_workspace_bytes(big, B.opts()) == 0
    assert "L <= 362" in B.cg_last_error()
    assert time.perf_counter() - t0 < 5.0


@pytest.mark.parametrize("L,r_max", [(16, 3), (10, 4), (30, 2), (36, 5)])
def test_workspace_plan_counts_the_random_site_geometry(libcg, L, r_max):
    # a random-site replica adds its positions (2 N doubles), the N x N
    # coupling matrix, a 64-byte guide record per site and per pair an
    # 8-byte record (running weight + partner) and a 16-byte one (1/r + E dx);
    # the pair count is the oracle's, whose full scan over every pair checks
    # the library's cell-list search (L / (r_max + 1) cells per axis; fewer
    # than 3 at L = 10, r_max = 4, where the library scans every pair too)
    import oracle
    from paper_1407_5026_gb300 import binding as B
    up = lambda b: (b + 255) // 256 * 256
    p = dict(L=L, r_max=r_max, xi=1.0, seed=5, replica=2)
    rnd = B.cg_workspace_bytes([B.desc(sites=B.CG_SITES_RANDOM, **p)], B.opts())
    lat = B.cg_workspace_bytes([B.desc(**p)], B.opts())
    cnt = len(oracle.Chain(L, r_max=r_max, xi=1.0, seed=5, replica=2,
                           random_sites=True).pairs()[1])
    N = L * L
    assert cnt > 0
    assert rnd - lat == 2 * up(N * 8) + up(N * N * 8) + up(N * 64) + up(cnt * 8) + up(cnt * 16)


def test_site_positions_checks_its_arguments_on_host(libcg):
    from paper_1407_5026_gb300 import binding as B
    with pytest.raises(B.CgError, match="null handle"):
        B.cg_site_positions(None, 0, n_sites=4)
