"""The C-ABI library builds, loads and exports every symbol include/ader.h declares;
host-only entry points behave (no GPU needed: ader_init and the table queries
allocate no device memory).  The library's operator tables (Golub-Welsch nodes,
barycentric basis, quadrature) are cross-checked against the oracle's (Newton
nodes, exact monomial integrals): two independent constructions of Sec. 1.1.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2409_12483_gb300 as pkg
    return pkg.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "ader.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ader_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    import paper_2409_12483_gb300 as pkg
    names = header_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(pkg.exported_symbols()) == names


def test_library_is_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    from paper_2409_12483_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_init_rejects_bad_arguments(lib):
    from paper_2409_12483_gb300.capi import Mesh, default_options
    opt = default_options()
    ctx = C.c_void_p()
    bad = [
        (Mesh(0, 0.0, 1.0), 2, 0),     # empty mesh
        (Mesh(-5, 0.0, 1.0), 2, 0),
        (Mesh(10, 1.0, 1.0), 2, 0),    # zero length
        (Mesh(10, 0.0, 1.0), 8, 0),    # degree above 7
        (Mesh(10, 0.0, 1.0), -1, 0),
        (Mesh(10, 0.0, 1.0), 3, 1),    # WENO needs an even degree 2 or 4
        (Mesh(10, 0.0, 1.0), 2, 7),    # unknown scheme
    ]
    for mesh, deg, scheme in bad:
        rc = lib.ader_init(C.byref(mesh), deg, scheme, C.byref(opt), C.byref(ctx))
        assert rc == 1, (mesh.n_cells, deg, scheme)
        assert not ctx.value
    o2 = default_options(fp64_sweeps=0, precision=1)
    rc = lib.ader_init(C.byref(Mesh(10, 0.0, 1.0)), 2, 0, C.byref(o2), C.byref(ctx))
    assert rc == 1


def test_cfl_mode_option(lib):
    """cfl_mode 1 (lambda over the nodal values) is a 1D DG Euler option without
    the limiter; elsewhere, and for unknown modes, ader_init refuses it."""
    from paper_2409_12483_gb300.capi import Mesh, Mesh2D, Mesh3D, default_options
    assert default_options().cfl_mode == 0
    ctx = C.c_void_p()
    m = Mesh(10, 0.0, 1.0)
    for scheme, deg, kw in [(0, 3, {}), (0, 0, {}), (0, 5, {"precision": "incr"}),
                            (0, 4, {"bc": "outflow"})]:
        o = default_options(cfl_mode="nodal", **kw)
        assert lib.ader_init(C.byref(m), deg, scheme, C.byref(o), C.byref(ctx)) == 0
        lib.ader_destroy(ctx)
    for scheme, deg, kw in [(1, 4, {}), (0, 3, {"limiter": 1}), (0, 3, {"system": "reacting"}),
                            (0, 3, {"system": "tracer"})]:
        o = default_options(cfl_mode=1, **kw)
        assert lib.ader_init(C.byref(m), deg, scheme, C.byref(o), C.byref(ctx)) == 1, (scheme, kw)
        assert not ctx.value
    o = default_options(cfl_mode=2)
    assert lib.ader_init(C.byref(m), 3, 0, C.byref(o), C.byref(ctx)) == 1
    o = default_options(cfl_mode=1)
    assert lib.ader_init_2d(C.byref(Mesh2D(4, 4, 0.0, 1.0, 0.0, 1.0)), 2, C.byref(o),
                            C.byref(ctx)) == 1
    assert lib.ader_init_3d(C.byref(Mesh3D(2, 2, 2, 0.0, 1.0, 0.0, 1.0, 0.0, 1.0)), 2,
                            C.byref(o), C.byref(ctx)) == 1


def test_sizes_and_coordinates(lib):
    from paper_2409_12483_gb300.capi import Mesh, default_options
    opt = default_options()
    for scheme, deg, per in [(0, 5, 6), (1, 4, 1)]:
        ctx = C.c_void_p()
        assert lib.ader_init(C.byref(Mesh(37, -1.0, 2.0)), deg, scheme, C.byref(opt),
                             C.byref(ctx)) == 0
        assert lib.ader_state_count(ctx) == 37 * per * 3
        assert lib.ader_predictor_count(ctx) == 37 * (deg + 1) ** 2 * 3
        assert lib.ader_workspace_bytes(ctx) >= 8 * 37 * (deg + 1) * 3
        x = np.zeros(37 * per)
        assert lib.ader_node_coords(ctx, x.ctypes.data_as(C.c_void_p), x.size) == 0
        assert lib.ader_node_coords(ctx, x.ctypes.data_as(C.c_void_p), x.size - 1) == 1
        assert np.all(np.diff(x) > 0) and x[0] > -1.0 and x[-1] < 2.0
        # calls that need a bound workspace say so instead of touching the GPU
        assert lib.ader_step(ctx, None, None, 0.1) in (1, 7)
        lib.ader_destroy(ctx)


@pytest.mark.parametrize("N", range(0, 8))
def test_library_tables_match_oracle(lib, oracle_mod, N):
    from paper_2409_12483_gb300.capi import Mesh, default_options
    ctx = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(4, 0.0, 1.0)), N, 0, C.byref(default_options()),
                         C.byref(ctx)) == 0
    o = oracle_mod.Oracle(N)
    n = N + 1

    def get(name, size):
        out = np.zeros(size)
        assert lib.ader_get_table(ctx, name.encode(), out.ctypes.data_as(C.c_void_p), size) == 0
        return out

    for name in ("xi", "w", "psi0", "psi1"):
        np.testing.assert_allclose(get(name, n), o.table(name), rtol=0, atol=2e-15, err_msg=name)
    for name, oname in (("kt", "kt"), ("kap", "kap"), ("dphi", "dphi"), ("dtil", "dt_m")):
        ref = o.table(oname)
        np.testing.assert_allclose(get(name, n * n).reshape(n, n), ref, rtol=0,
                                   atol=4e-15 * max(1.0, np.abs(ref).max()), err_msg=name)
    Ns = 2 * N + 1
    np.testing.assert_allclose(get("P", Ns * n).reshape(Ns, n), o.table("P"), rtol=0, atol=4e-15)
    # k~ in even/odd form, applied the way the predictor applies it, gives the
    # oracle's k~ f (the GL nodes are symmetric, so k~ is centro-antisymmetric)
    H, h = (n + 1) // 2, n // 2
    ka = get("ksa", H * H).reshape(H, H)
    kb = get("ksb", H * H).reshape(H, H)
    kt = o.table("kt")
    for seed in range(3):
        f = np.random.default_rng(100 * N + seed).standard_normal(n)
        e = np.array([f[q] + f[n - 1 - q] for q in range(h)] + ([f[h]] if H > h else []))
        od = np.array([f[q] - f[n - 1 - q] for q in range(h)])
        g = np.empty(n)
        for p in range(h):
            S, T = ka[p, :H] @ e, kb[p, :h] @ od
            g[p], g[n - 1 - p] = S + T, T - S
        if H > h:
            g[h] = kb[h, :h] @ od
        np.testing.assert_allclose(g, kt @ f, rtol=0,
                                   atol=1e-14 * np.abs(kt).sum(1).max() * np.abs(f).max())
    lib.ader_destroy(ctx)


def test_server_rejects_bad_options_and_requests(lib):
    from paper_2409_12483_gb300.capi import Request, ServerOpts
    o = ServerOpts()
    assert lib.ader_server_default_options(C.byref(o)) == 0
    srv = C.c_void_p()
    assert lib.ader_server_create(C.byref(o), C.byref(srv)) == 1  # no pool
    o.pool_dev = 256
    o.pool_bytes = 1 << 20
    o.ticks_per_round = 3  # must be even
    assert lib.ader_server_create(C.byref(o), C.byref(srv)) == 1
    assert lib.ader_server_request_bytes(5, 1000) >= 1000 * 6 * 3 * 8 * 2 + 1000 * 54 * 8
    assert lib.ader_server_request_bytes(8, 10) == 0


def test_tuning_validation_without_gpu(lib):
    from paper_2409_12483_gb300.capi import Mesh, Tuning, default_options
    ctx = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(100, 0.0, 1.0)), 7, 0, C.byref(default_options()),
                         C.byref(ctx)) == 0
    t = Tuning()
    assert lib.ader_get_tuning(ctx, C.byref(t)) == 0
    # a small mesh defaults to half-size tiles, a large one to 32 / 64 cells
    assert (t.predict_cells_per_block, t.face_cells_per_block) == (16, 32)
    assert t.graph_steps >= 2 and t.graph_steps % 2 == 0
    big = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(100_000, 0.0, 1.0)), 2, 0, C.byref(default_options()),
                         C.byref(big)) == 0
    assert lib.ader_get_tuning(big, C.byref(t)) == 0
    assert (t.predict_cells_per_block, t.face_cells_per_block) == (32, 64)
    lib.ader_destroy(big)
    # 16-cell tiles are accepted at every degree (a partial last warp for even N)
    even = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(100, 0.0, 1.0)), 2, 0, C.byref(default_options()),
                         C.byref(even)) == 0
    assert lib.ader_set_tuning(even, C.byref(Tuning(16, 64, 8, 0.0, 0.0, 0.0))) == 0
    assert lib.ader_set_tuning(even, C.byref(Tuning(64, 64, 8, 0.0, 0.0, 0.0))) == 0
    lib.ader_destroy(even)
    for cpb, cpf, k in [(64, 64, 8), (8, 64, 8), (32, 48, 8), (32, 64, 7), (32, 64, 0)]:
        bad = Tuning(cpb, cpf, k, 0.0, 0.0, 0.0)  # 64 cells x 8 nodes is too big at N = 7
        assert lib.ader_set_tuning(ctx, C.byref(bad)) == 1
    ok = Tuning(32, 32, 16, 0.0, 0.0, 0.0)
    assert lib.ader_set_tuning(ctx, C.byref(ok)) == 0
    assert lib.ader_get_tuning(ctx, C.byref(t)) == 0 and t.face_cells_per_block == 32
    lib.ader_destroy(ctx)


def test_per_degree_helpers_are_not_merged_across_degrees():
    """Launch helpers compiled once per degree must have internal linkage: a weak
    (mergeable) definition would make every degree launch one degree's kernels."""
    import shutil
    import subprocess
    from paper_2409_12483_gb300 import build
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-C", build.LIB], capture_output=True, text=True).stdout
    weak = [l for l in out.splitlines()
            if l.split()[1:2] and l.split()[1] in ("W", "V", "u")
            and ("ader::" in l) and ("launch" in l or "prepare" in l)]
    assert not weak, weak[:5]


@pytest.mark.parametrize("N", [2, 4])
def test_weno_monomial_tables_reproduce_polynomials(lib, N):
    """The WENO kernel's tables, applied as the kernel applies them: from the
    exact cell averages of a degree-N polynomial, every stencil's monomial
    coefficients (t = 2 xi - 1 in cell i) are the polynomial's own, and the
    nodal table gives its values at the GL nodes (reconstruction is exact for
    polynomials of degree <= N whatever the weights)."""
    from paper_2409_12483_gb300.capi import Mesh, default_options
    ctx = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(16, 0.0, 1.0)), N, 1, C.byref(default_options()),
                         C.byref(ctx)) == 0
    n = N + 1

    def get(name, size):
        out = np.zeros(size)
        assert lib.ader_get_table(ctx, name.encode(), out.ctypes.data_as(C.c_void_p), size) == 0
        return out

    amono = get("wamono", 3 * n * n).reshape(3, n, n)
    vnod = get("wvnod", n * n).reshape(n, n)
    xi = get("xi", n)
    P = np.polynomial.Polynomial
    for seed in range(3):
        p = P(np.random.default_rng(seed).standard_normal(n))   # in xi, cell i = [0, 1]
        Pint = p.integ()
        avg = {j: Pint(j + 1) - Pint(j) for j in range(-N, N + 1)}
        a_ref = p(P([0.5, 0.5])).coef                             # xi = (t + 1) / 2
        for S, shift in enumerate((-N // 2, -N, 0)):
            a = amono[S] @ np.array([avg[shift + k] for k in range(n)])
            np.testing.assert_allclose(a, a_ref, rtol=0, atol=1e-11 * np.abs(a_ref).max())
        np.testing.assert_allclose(vnod @ a_ref, p(xi), rtol=0, atol=1e-13 * np.abs(p(xi)).max())
    lib.ader_destroy(ctx)


def test_reacting_system_options_and_sizes(lib):
    """The reacting system: DG + FP64 only; M = 5 variables in the state and
    predictor sizes; an unknown system id is rejected."""
    from paper_2409_12483_gb300.capi import Mesh, default_options
    N, nc = 3, 10
    ctx = C.c_void_p()
    o = default_options(system="reacting", omega=2.0)
    assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), N, 0, C.byref(o), C.byref(ctx)) == 0
    assert lib.ader_state_count(ctx) == nc * (N + 1) * 5
    assert lib.ader_predictor_count(ctx) == nc * (N + 1) ** 2 * 5
    e = default_options()
    eul = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), N, 0, C.byref(e), C.byref(eul)) == 0
    # trace records grow from 3 x 3 (N+1) to 3 x 5 (N+1) doubles per cell
    assert lib.ader_workspace_bytes(ctx) > lib.ader_workspace_bytes(eul)
    lib.ader_destroy(ctx)
    lib.ader_destroy(eul)
    for kw, scheme, deg in ((dict(system="reacting"), 1, 4),             # FV
                            (dict(system="reacting", precision="ff"), 0, 3),
                            (dict(system="reacting", precision="fp32"), 0, 3),
                            (dict(system=7), 0, 3),
                            (dict(system="reacting", omega=float("nan")), 0, 3)):
        bad = C.c_void_p()
        assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), deg, scheme,
                             C.byref(default_options(**kw)), C.byref(bad)) == 1, kw


def test_boundary_and_limiter_options(lib, oracle_mod):
    """Outflow and the limiter are DG options (the limiter for the Euler system and
    N >= 1, modes 1 and 2); the limiter adds its per-cell buffers to the
    workspace; the library's R is the oracle's pseudo-inverse of P."""
    from paper_2409_12483_gb300.capi import Mesh, default_options
    nc = 10
    ok = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), 3, 0,
                         C.byref(default_options(bc="outflow", limiter=1)), C.byref(ok)) == 0
    plain = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), 3, 0, C.byref(default_options()),
                         C.byref(plain)) == 0
    assert lib.ader_workspace_bytes(ok) > lib.ader_workspace_bytes(plain)
    R = np.zeros(4 * 7)
    assert lib.ader_get_table(ok, b"R", R.ctypes.data_as(C.c_void_p), R.size) == 0
    np.testing.assert_allclose(R.reshape(4, 7), oracle_mod.Oracle(3).r_matrix(), rtol=0, atol=1e-13)
    lib.ader_destroy(ok)
    lib.ader_destroy(plain)
    every = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), 1, 0, C.byref(default_options(limiter=2)),
                         C.byref(every)) == 0
    lib.ader_destroy(every)
    for kw, scheme, deg in ((dict(bc="outflow"), 1, 4), (dict(limiter=1), 1, 4),
                            (dict(limiter=1, system="reacting"), 0, 3), (dict(bc=5), 0, 3),
                            (dict(limiter=3), 0, 3), (dict(limiter=-1), 0, 3),
                            (dict(limiter=1), 0, 0), (dict(limiter=2), 0, 0),
                            (dict(limiter=1, nad_eps=-1.0), 0, 3)):
        bad = C.c_void_p()
        assert lib.ader_init(C.byref(Mesh(nc, 0.0, 1.0)), deg, scheme,
                             C.byref(default_options(**kw)), C.byref(bad)) == 1, kw


def test_init_2d_options_and_sizes(lib):
    """ader_init_2d: DG Euler FP64 periodic without limiter only; the state is
    nx ny (N+1)^2 4 doubles; the 1D-only node coordinates are refused."""
    from paper_2409_12483_gb300.capi import Mesh2D, default_options
    ctx = C.c_void_p()
    assert lib.ader_init_2d(C.byref(Mesh2D(6, 5, 0.0, 1.0, 0.0, 2.0)), 4,
                            C.byref(default_options()), C.byref(ctx)) == 0
    assert lib.ader_state_count(ctx) == 6 * 5 * 25 * 4
    assert lib.ader_predictor_count(ctx) == 6 * 5 * 125 * 4
    assert lib.ader_workspace_bytes(ctx) > 2 * 8 * lib.ader_state_count(ctx)
    x = np.zeros(30 * 5)
    assert lib.ader_node_coords(ctx, x.ctypes.data_as(C.c_void_p), x.size) == 1
    lib.ader_destroy(ctx)
    for kw in (dict(precision="fp32"), dict(system="reacting"), dict(bc="outflow"), dict(limiter=1)):
        bad = C.c_void_p()
        assert lib.ader_init_2d(C.byref(Mesh2D(4, 4, 0.0, 1.0, 0.0, 1.0)), 2,
                                C.byref(default_options(**kw)), C.byref(bad)) == 1, kw
    for mesh in (Mesh2D(0, 4, 0.0, 1.0, 0.0, 1.0), Mesh2D(4, 4, 0.0, 1.0, 1.0, 1.0)):
        bad = C.c_void_p()
        assert lib.ader_init_2d(C.byref(mesh), 2, None, C.byref(bad)) == 1
    bad = C.c_void_p()
    assert lib.ader_init_2d(C.byref(Mesh2D(4, 4, 0.0, 1.0, 0.0, 1.0)), 8, None, C.byref(bad)) == 1


def test_init_3d_options_and_sizes(lib):
    """ader_init_3d: degrees 0..7, DG Euler FP64 periodic without limiter; the state
    is nx ny nz (N+1)^3 5 doubles"""
    from paper_2409_12483_gb300.capi import Mesh3D, default_options
    ctx = C.c_void_p()
    assert lib.ader_init_3d(C.byref(Mesh3D(4, 3, 2, 0, 1, 0, 1, 0, 2)), 3,
                            C.byref(default_options()), C.byref(ctx)) == 0
    assert lib.ader_state_count(ctx) == 24 * 64 * 5
    assert lib.ader_predictor_count(ctx) == 24 * 256 * 5
    lib.ader_destroy(ctx)
    ok = C.c_void_p()
    assert lib.ader_init_3d(C.byref(Mesh3D(2, 2, 2, 0, 1, 0, 1, 0, 1)), 7, None, C.byref(ok)) == 0
    assert lib.ader_state_count(ok) == 8 * 512 * 5
    lib.ader_destroy(ok)
    for deg in (8, -1):
        bad = C.c_void_p()
        assert lib.ader_init_3d(C.byref(Mesh3D(2, 2, 2, 0, 1, 0, 1, 0, 1)), deg, None,
                                C.byref(bad)) == 1
    for kw in (dict(limiter=1), dict(bc="outflow"), dict(precision="ff")):
        bad = C.c_void_p()
        assert lib.ader_init_3d(C.byref(Mesh3D(2, 2, 2, 0, 1, 0, 1, 0, 1)), 2,
                                C.byref(default_options(**kw)), C.byref(bad)) == 1, kw
    bad = C.c_void_p()
    assert lib.ader_init_3d(C.byref(Mesh3D(2, 2, 0, 0, 1, 0, 1, 0, 1)), 2, None, C.byref(bad)) == 1


def test_tracer_system_options(lib):
    """the non-conservative tracer system: DG, FP64, periodic; 4 variables per node"""
    from paper_2409_12483_gb300.capi import Mesh, default_options
    ctx = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(10, 0.0, 1.0)), 3, 0,
                         C.byref(default_options(system="tracer")), C.byref(ctx)) == 0
    assert lib.ader_state_count(ctx) == 10 * 4 * 4
    lib.ader_destroy(ctx)
    for kw, scheme in ((dict(system="tracer", bc="outflow"), 0), (dict(system="tracer"), 1),
                       (dict(system="tracer", precision="ff"), 0),
                       (dict(system="tracer", limiter=1), 0)):
        bad = C.c_void_p()
        assert lib.ader_init(C.byref(Mesh(10, 0.0, 1.0)), 4 if scheme else 3, scheme,
                             C.byref(default_options(**kw)), C.byref(bad)) == 1, kw


def test_shard_init_layout_and_validation(lib):
    """ader_init_shard: halo width (DG 1, WENO-FV N + 1), the extended array's
    size, its node coordinates equal to the global mesh's, and the rejected
    configurations (outflow, limiter, blocks smaller than the stencil)."""
    from paper_2409_12483_gb300.capi import Mesh, ShardInfo, default_options
    opt = default_options()
    g = Mesh(40, -1.0, 3.0)
    for scheme, N, H, per in [(0, 3, 1, 4 * 3), (1, 4, 5, 3), (1, 2, 3, 3)]:
        ctx = C.c_void_p()
        assert lib.ader_init_shard(C.byref(g), 10, 17, N, scheme, C.byref(opt), C.byref(ctx)) == 0
        info = ShardInfo()
        assert lib.ader_shard_info(ctx, C.byref(info)) == 0
        assert (info.first_cell, info.n_local, info.n_global, info.halo_cells) == (10, 17, 40, H)
        assert info.values_per_cell == per
        assert lib.ader_state_count(ctx) == (17 + 2 * H) * per
        # coordinates of the extended array = the global mesh's cells 10-H .. 27+H
        k = per // 3
        x = np.zeros((17 + 2 * H) * k)
        assert lib.ader_node_coords(ctx, x.ctypes.data_as(C.c_void_p), x.size) == 0
        full = C.c_void_p()
        assert lib.ader_init(C.byref(g), N, scheme, C.byref(opt), C.byref(full)) == 0
        xg = np.zeros(40 * k)
        assert lib.ader_node_coords(full, xg.ctypes.data_as(C.c_void_p), xg.size) == 0
        assert np.allclose(x[:H * k], xg[(10 - H) * k:10 * k], rtol=0, atol=1e-13)
        assert np.allclose(x[H * k:(17 + H) * k], xg[10 * k:27 * k], rtol=0, atol=1e-13)
        lib.ader_destroy(full)
        # a shard has no device-resident time loop; calls that need a workspace say so
        assert lib.ader_solve(ctx, None, 1.0, 0, None, None) in (1, 7)
        lib.ader_destroy(ctx)
    plain = C.c_void_p()
    assert lib.ader_init(C.byref(g), 3, 0, C.byref(opt), C.byref(plain)) == 0
    assert lib.ader_shard_info(plain, C.byref(ShardInfo())) == 1
    lib.ader_destroy(plain)
    ctx = C.c_void_p()
    bad = [(g, 35, 10, 3, 0, opt),                         # block beyond the mesh
           (g, -1, 10, 3, 0, opt), (g, 0, 0, 3, 0, opt),
           (g, 0, 3, 4, 1, opt),                           # WENO5 block smaller than N
           (g, 0, 10, 3, 0, default_options(bc=1)),        # outflow
           (g, 0, 10, 3, 0, default_options(limiter=1))]
    for mesh, first, nl, N, scheme, o in bad:
        assert lib.ader_init_shard(C.byref(mesh), first, nl, N, scheme, C.byref(o),
                                   C.byref(ctx)) == 1, (first, nl, N, scheme)
        assert not ctx.value


def test_resident_state_calls_need_a_workspace(lib):
    from paper_2409_12483_gb300.capi import Mesh, default_options
    opt = default_options()
    ctx = C.c_void_p()
    assert lib.ader_init(C.byref(Mesh(12, 0.0, 1.0)), 2, 0, C.byref(opt), C.byref(ctx)) == 0
    u = np.zeros(12 * 3 * 3)
    ptr = u.ctypes.data_as(C.c_void_p)
    assert lib.ader_set_state(ctx, ptr, u.size, 0) == 7
    assert lib.ader_get_state(ctx, ptr, u.size, 0) == 7
    assert lib.ader_state_step(ctx, 0.1, None) == 7
    assert lib.ader_state_solve(ctx, 1.0, 0, None, None) == 7
    assert lib.ader_get_predictor(ctx, 0.1, ptr, 12 * 9 * 3) == 7
    t = C.c_double(0.0)
    assert lib.ader_get_state_time(ctx, C.byref(t)) == 7
    lib.ader_destroy(ctx)
