"""The C ABI on the host (no GPU needed): libfwi.so loads, exports every entry
point include/fwi.h declares, and fwi_plan_create validates its arguments
(host-only call) with the documented error codes."""
import ctypes
import dataclasses
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fwi.h")
LIB = os.path.join(ROOT, "paper_2603_16393_gb300", "libfwi.so")


@pytest.fixture(scope="module")
def api():
    if not os.path.exists(LIB):
        from paper_2603_16393_gb300 import _build
        _build.build_library()
    from paper_2603_16393_gb300 import api as A
    return A


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FWI_API\s+[^;(]*?\b(fwi_\w+)\s*\(", text)))


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("fwi_forward", "fwi_w2_misfit", "fwi_adjoint_grad", "fwi_guided_step",
              "fwi_w2_prepare", "fwi_plan_create", "fwi_plan_sizes", "fwi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(api):
    lib = ctypes.CDLL(LIB)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert api.fwi_version() == 11400


def _prob(api, **kw):
    base = dict(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3,
                src_iz=(0,) * 5, src_ix=(0, 17, 34, 52, 69), rec_iz=(0,) * 70,
                rec_ix=tuple(range(70)), v_max=4500.0, batch=3)
    base.update(kw)
    return api.Problem(**base)


def test_plan_sizes_of_the_benchmark_problem(api):
    h = api.fwi_plan_create(_prob(api), api.W2Params())
    ws, ctx, snap = api.fwi_plan_sizes(h)
    B, ns, nr, nt, NZ, NX = 3, 5, 70, 1000, 110, 150
    # one record plane per step: 110 rows at the compile-time pitch 160 of
    # the fast propagators (the 10 pad columns are never touched)
    assert snap == B * ns * nt * NZ * 160 * 4
    assert ws >= 256 + B * ns * nr * 4 + B * ns * 70 * 70 * 4
    assert ctx >= B * ns * nr * (nt * 4 + 1000 * 8)


def test_plan_of_a_grid_beyond_shared_memory_uses_the_tiled_fields(api):
    # 256 x 256 with a 40-cell layer: 296 x 336 padded cells, fields of pitch 336
    B, ns, nt = 2, 16, 200
    prob = _prob(api, nz=256, nx=256, nt=nt, batch=B, src_iz=(0,) * ns,
                 src_ix=tuple(range(0, 256, 16)), rec_iz=(0,) * 256, rec_ix=tuple(range(256)))
    h = api.fwi_plan_create(dataclasses.replace(prob, kernels=api.KERNELS_TILED), api.W2Params())
    assert api.fwi_plan_kernels(h) == api.KERNELS_TILED
    ws, ctx, snap = api.fwi_plan_sizes(h)
    NZ, NX, NXp = 296, 336, 336
    assert snap == B * ns * nt * NZ * NXp * 4
    assert ws >= 6 * B * ns * NZ * NXp * 4 + 2 * B * NZ * NXp * 4
    # the automatic choice for this grid: column pairs, a cluster of 8 CTAs of
    # 40 rows (four 10-row strips of 168 column pairs; the last CTA holds 16
    # grid rows); record rows at the cluster kernels' pitch 340
    h = api.fwi_plan_create(prob, api.W2Params())
    assert api.fwi_plan_kernels(h) == api.KERNELS_CLUSTER
    assert api.fwi_plan_sizes(h)[2] == B * ns * nt * (8 * 40) * 340 * 4
    # single columns: 8 CTAs of 38 rows (two 19-row strips)
    h = api.fwi_plan_create(dataclasses.replace(prob, shape=api.SHAPE_CLUSTER_RS19),
                            api.W2Params())
    assert api.fwi_plan_kernels(h) == api.KERNELS_CLUSTER
    assert api.fwi_plan_sizes(h)[2] == B * ns * nt * (8 * 38) * 340 * 4
    # odd padded width: rows padded to a multiple of 4 floats
    prob = _prob(api, nz=200, nx=301, nt=nt, batch=1, src_ix=(0, 75, 150, 225, 300),
                 rec_iz=(0,) * 301, rec_ix=tuple(range(301)))
    h = api.fwi_plan_create(prob, api.W2Params())
    assert api.fwi_plan_kernels(h) == api.KERNELS_TILED     # 381 columns: wider than a cluster's rows
    assert api.fwi_plan_sizes(h)[2] == 5 * nt * 240 * 384 * 4
    # with checkpoints: two compact NZ x NX grids per slot
    h = api.fwi_plan_create(_prob(api, nz=256, nx=256, nt=nt, batch=B, src_iz=(0,) * ns,
                                  src_ix=tuple(range(0, 256, 16)), rec_iz=(0,) * 256,
                                  rec_ix=tuple(range(256)), checkpoint_every=32),
                            api.W2Params())
    assert api.fwi_plan_sizes(h)[2] == 7 * B * ns * 2 * NZ * NX * 4


@pytest.mark.parametrize("K", [32, 7, 1, 1000, 5000])
def test_plan_sizes_with_checkpoints(api, K):
    # checkpoint_every = K: ceil(nt/K) slots of two padded grids per (model,
    # shot) instead of nt record planes; the workspace gains one K-plane
    # segment of the record, the adjoint state (three grids) and one float
    B, ns, nt, NZ, NX = 3, 5, 1000, 110, 150
    h0 = api.fwi_plan_create(_prob(api), api.W2Params())
    ws0, ctx0, snap0 = api.fwi_plan_sizes(h0)
    h = api.fwi_plan_create(_prob(api, checkpoint_every=K), api.W2Params())
    ws, ctx, snap = api.fwi_plan_sizes(h)
    Ke = min(K, nt)
    assert snap == -(-nt // Ke) * B * ns * 2 * NZ * NX * 4
    assert ctx == ctx0
    seg = B * ns * Ke * NZ * 160 * 4
    state = B * ns * 3 * NZ * NX * 4 + B * ns * 4
    assert seg + state <= ws - ws0 <= seg + state + 3 * 256
    if K == 32:
        assert snap0 / snap > 16     # K/2 x (record pitch 160 / 150)


@pytest.mark.parametrize("kw,code", [
    (dict(v_max=9000.0), 2),                 # CFL: 9000*1e-3*sqrt(2)/10 = 1.27 > 0.866
    (dict(dt=2e-3, v_max=4500.0), 2),        # 0.636*2 = 1.27
    (dict(nz=0), 1),
    (dict(nt=1), 1),
    (dict(dx=-1.0), 1),
    (dict(src_iz=(0, 0), src_ix=(0, 70)), 1),  # outside the grid
    (dict(rec_iz=(0, 70), rec_ix=(1, 2)), 1),
    (dict(batch=0), 1),
    (dict(top_bc=2), 1),
    (dict(checkpoint_every=-1), 1),
    (dict(refl_R=0.0), 1),
    (dict(nx=1200, batch=13108), 3),         # tiled grid, batch x ns > 65535 (its grid z)
    (dict(rec_iz=(0, 1), rec_ix=(5, 5)), 3),  # two receivers in one column strip
])
def test_plan_rejects_invalid_problems(api, kw, code):
    with pytest.raises(api.FwiError) as e:
        api.fwi_plan_create(_prob(api, **kw), api.W2Params())
    assert e.value.code == code
    assert api.fwi_last_error() != ""


def test_plan_rejects_bad_w2_params(api):
    for w2 in (api.W2Params(n_xi=1), api.W2Params(k=-1.0), api.W2Params(eps_density=-1e-9)):
        with pytest.raises(api.FwiError) as e:
            api.fwi_plan_create(_prob(api), w2)
        assert e.value.code == 1


def test_cfl_limit_is_sqrt3_over_2(api):
    # exactly at the bound passes, just above fails
    vmax_ok = 0.866 / (1e-3 * (2 ** 0.5) / 10.0)
    api.fwi_plan_create(_prob(api, v_max=vmax_ok * 0.9999), api.W2Params())
    with pytest.raises(api.FwiError):
        api.fwi_plan_create(_prob(api, v_max=vmax_ok * 1.001), api.W2Params())


def test_binding_fails_loudly_without_library(tmp_path):
    # the binding must not fall back to anything when libfwi.so is absent
    import subprocess
    import sys
    code = ("import sys, os; sys.path.insert(0, %r); import paper_2603_16393_gb300.api as A"
            % str(tmp_path))
    pkg = tmp_path / "paper_2603_16393_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "api.py"):
        (pkg / f).write_text(open(os.path.join(ROOT, "paper_2603_16393_gb300", f)).read())
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode != 0 and "libfwi.so is missing" in r.stderr


def test_space_order_and_its_cfl_bound(api):
    # 8th order: lambda = 205/72 + 2 (8/5 + 1/5 + 8/315 + 1/560) = 6.50159, bound 2/sqrt(lambda)
    lam = 205 / 72 + 2 * (8 / 5 + 1 / 5 + 8 / 315 + 1 / 560)
    bound = 2 / lam ** 0.5
    vmax = bound / (1e-3 * 2 ** 0.5 / 10.0)
    api.fwi_plan_create(_prob(api, v_max=vmax * 0.9999, space_order=8), api.W2Params())
    with pytest.raises(api.FwiError) as e:
        api.fwi_plan_create(_prob(api, v_max=vmax * 1.001, space_order=8), api.W2Params())
    assert e.value.code == 2
    # the same v_max is fine at 4th order (bound sqrt(3)/2)
    api.fwi_plan_create(_prob(api, v_max=vmax * 1.001), api.W2Params())
    with pytest.raises(api.FwiError) as e:
        api.fwi_plan_create(_prob(api, space_order=6), api.W2Params())
    assert e.value.code == 1
    # an 8th-order plan of a 70x70 grid runs on the tiled fields (row pitch 152)
    h = api.fwi_plan_create(_prob(api, space_order=8), api.W2Params())
    assert api.fwi_plan_sizes(h)[2] == 3 * 5 * 1000 * 110 * 152 * 4


def test_kernel_family_selection(api):
    K = api
    # automatic: 70 x 70 (110 x 150 padded) on the resident kernels
    assert K.fwi_plan_kernels(K.fwi_plan_create(_prob(api), K.W2Params())) == K.KERNELS_RESIDENT
    for fam in (K.KERNELS_RESIDENT, K.KERNELS_TILED, K.KERNELS_CLUSTER):
        h = K.fwi_plan_create(_prob(api, kernels=fam), K.W2Params())
        assert K.fwi_plan_kernels(h) == fam
    # a cluster plan's record: ceil(110 / 8) = 14 rows a CTA round up to two
    # 10-row strips of column pairs, so 6 CTAs of 20 rows: 120 rows at the
    # pitch 340; with 13-row single-column strips 5 CTAs of 26 rows
    h = K.fwi_plan_create(_prob(api, kernels=K.KERNELS_CLUSTER), K.W2Params())
    assert K.fwi_plan_sizes(h)[2] == 3 * 5 * 1000 * 120 * 340 * 4
    h = K.fwi_plan_create(_prob(api, kernels=K.KERNELS_CLUSTER, shape=K.SHAPE_CLUSTER_RS13),
                          K.W2Params())
    assert K.fwi_plan_sizes(h)[2] == 3 * 5 * 1000 * 130 * 340 * 4
    # a grid of 10 rows or fewer would need a cluster of one CTA
    with pytest.raises(K.FwiError) as e:
        K.fwi_plan_create(_prob(api, nz=7, nb=3, src_iz=(0,), src_ix=(0,),
                                kernels=K.KERNELS_CLUSTER), K.W2Params())
    assert e.value.code == 3
    # checkpointed or 8th-order plans of a cluster-sized grid run tiled
    for kw in (dict(checkpoint_every=32), dict(space_order=8)):
        assert K.fwi_plan_kernels(K.fwi_plan_create(_prob(api, nz=200, **kw), K.W2Params())) \
            == K.KERNELS_TILED
    big = dict(nz=256, nx=256, src_iz=(0,), src_ix=(0,), rec_iz=(0,) * 256,
               rec_ix=tuple(range(256)))
    bad = [
        (dict(big, kernels=K.KERNELS_RESIDENT), 3),          # 296 x 336 cells: not one CTA's
        (dict(kernels=K.KERNELS_CLUSTER, checkpoint_every=8), 3),
        (dict(kernels=K.KERNELS_CLUSTER, space_order=8), 3),
        (dict(kernels=K.KERNELS_RESIDENT, space_order=8), 3),
        (dict(nx=300, kernels=K.KERNELS_CLUSTER), 3),        # 380 padded columns
        (dict(kernels=5), 1),
        (dict(kernels=-1), 1),
    ]
    for kw, code in bad:
        with pytest.raises(K.FwiError) as e:
            K.fwi_plan_create(_prob(api, **kw), K.W2Params())
        assert e.value.code == code, kw


def test_cpml_plans():
    K = api = __import__("paper_2603_16393_gb300.api", fromlist=["api"])
    h = K.fwi_plan_create(_prob(api, absorber=K.ABSORBER_CPML), K.W2Params())
    assert K.fwi_plan_kernels(h) == K.KERNELS_CPML
    ws, _, snap = K.fwi_plan_sizes(h)
    B, ns, nt, NZ, NX = 3, 5, 1000, 110, 150
    assert snap == B * ns * nt * NZ * NX * 4          # record B^n, compact rows
    assert ws >= 12 * B * ns * NZ * NX * 4 + B * NZ * NX * 4
    for kw in (dict(top_bc=1), dict(checkpoint_every=16), dict(space_order=8),
               dict(kernels=K.KERNELS_RESIDENT), dict(kernels=K.KERNELS_CLUSTER),
               dict(rec_iz=(0, 0), rec_ix=(3, 3))):
        with pytest.raises(K.FwiError) as e:
            K.fwi_plan_create(_prob(api, absorber=K.ABSORBER_CPML, **kw), K.W2Params())
        assert e.value.code == 3, kw
    with pytest.raises(K.FwiError) as e:               # the CPML family needs the CPML absorber
        K.fwi_plan_create(_prob(api, kernels=K.KERNELS_CPML), K.W2Params())
    assert e.value.code == 3
    with pytest.raises(K.FwiError) as e:
        K.fwi_plan_create(_prob(api, absorber=2), K.W2Params())
    assert e.value.code == 1


def test_compute_entry_points_reject_null_and_bad_sizes_without_a_gpu():
    # argument checks run on the host before any CUDA call: every call below
    # returns FWI_ERR_INVALID_ARG (1) on a machine with no GPU at all
    K = __import__("paper_2603_16393_gb300.api", fromlist=["api"])
    lib = K._lib
    h = K.fwi_plan_create(_prob(K), K.W2Params())
    p = h.raw
    g = K._Guide(1.0, 0.1, 0.0, 0.5, 1e-4, 0.0, 0.0, 1.0)
    calls = [
        lambda: lib.fwi_forward(p, None, None, None, None, None),
        lambda: lib.fwi_forward(None, None, None, None, None, None),
        lambda: lib.fwi_w2_prepare(p, None, None, None),
        lambda: lib.fwi_w2_misfit(p, None, None, None, None, None, None, None),
        lambda: lib.fwi_adjoint_grad(p, None, None, None, None, None, None),
        lambda: lib.fwi_w2_misfit_static(p, None, None, None, None, None, None),
        lambda: lib.fwi_l2_misfit(p, None, None, 1.0, None, None, None),
        lambda: lib.fwi_guided_step(0, 4, 4, ctypes.byref(g), *([None] * 7)),
        lambda: lib.fwi_guided_step(1, 4, 4, None, *([None] * 7)),
        lambda: lib.fwi_tv_grad(1, 4, 4, 0.1, 1.0, None, None, None, None, None),
        lambda: lib.fwi_tv_grad(0, 4, 4, 0.1, 1.0, None, None, None, None, None),
        lambda: lib.fwi_image_metrics(1, 4, 4, 1.0, None, None, None, None),
        lambda: lib.fwi_check(p, None, None),
        lambda: lib.fwi_plan_sizes(None, None, None, None),
        lambda: lib.fwi_plan_kernels(p, None),
    ]
    for i, call in enumerate(calls):
        assert call() == 1, i
        assert K.fwi_last_error() != ""


def test_group_create_rejects_bad_arguments_without_a_gpu():
    K = __import__("paper_2603_16393_gb300.api", fromlist=["api"])
    lib = K._lib
    h = K.fwi_plan_create(_prob(K), K.W2Params())
    out = ctypes.c_void_p()
    plans = (ctypes.c_void_p * 2)(h.raw, None)
    assert lib.fwi_group_create(plans, 0, ctypes.byref(out)) == 1
    assert lib.fwi_group_create(plans, 2, ctypes.byref(out)) == 1      # plan 1 is NULL
    assert lib.fwi_group_create(None, 1, ctypes.byref(out)) == 1
    assert lib.fwi_group_create(plans, 1, None) == 1
    nul = (ctypes.c_void_p * 1)(None)
    assert lib.fwi_group_gradient(None, *([nul] * 8), None) == 1


def test_coarse_problem_matches_the_oracle_twin(api):
    # the library's derivation of the low-fidelity problem against the
    # oracle's, on the benchmark geometry and on odd sizes and receiver counts
    from oracle import multifidelity as MF
    from oracle import oracle as O
    for kw in (dict(), dict(nz=33, nx=41, nb=7, nt=301, src_ix=(0, 20, 40), src_iz=(3, 0, 5),
                            rec_iz=tuple(range(9)), rec_ix=tuple(range(0, 41, 5)),
                            checkpoint_every=7)):
        fine = _prob(api, **kw)
        c = api.coarse_problem(fine)
        o = MF.coarse_problem(O.Problem(nz=fine.nz, nx=fine.nx, nb=fine.nb, nt=fine.nt,
                                        dz=fine.dz, dx=fine.dx, dt=fine.dt,
                                        src_iz=fine.src_iz, src_ix=fine.src_ix,
                                        rec_iz=fine.rec_iz, rec_ix=fine.rec_ix))
        assert (c.nz, c.nx, c.nb, c.nt) == (o.nz, o.nx, o.nb, o.nt)
        assert (c.dz, c.dx, c.dt) == (o.dz, o.dx, o.dt)
        assert list(c.src_iz) == list(o.src_iz) and list(c.src_ix) == list(o.src_ix)
        assert list(c.rec_iz) == list(o.rec_iz) and list(c.rec_ix) == list(o.rec_ix)
        assert c.checkpoint_every == ((fine.checkpoint_every + 1) // 2
                                      if fine.checkpoint_every else 0)
        assert (c.batch, c.f_peak, c.v_ref, c.v_max) == (fine.batch, fine.f_peak, fine.v_ref,
                                                         fine.v_max)
        api.fwi_plan_create(c, api.W2Params())   # a valid plan (freed with its handle)


def test_coarse_problem_rejects_short_runs(api):
    with pytest.raises(api.FwiError) as e:
        api.coarse_problem(_prob(api, nt=3))
    assert e.value.code == api.FWI_ERR_INVALID_ARG


def test_queue_rejects_plans_outside_the_column_pair_kernels(api):
    # an odd padded width (no column pairs) and a checkpointed plan: refused
    # before any CUDA call
    odd = api.fwi_plan_create(_prob(api, nx=69, src_ix=(0, 17, 34, 51, 68),
                                    rec_ix=tuple(range(69)), rec_iz=(0,) * 69), api.W2Params())
    ck = api.fwi_plan_create(_prob(api, checkpoint_every=32), api.W2Params())
    ok = api.fwi_plan_create(_prob(api), api.W2Params())
    vp = ctypes.c_void_p
    dummy = (vp * 2)(vp(256), vp(256))
    cnt = ctypes.c_void_p(256)
    for bad in (odd, ck):
        plans = (vp * 2)(ok.raw, bad.raw)
        rc = api._lib.fwi_queue_forward(plans, 2, dummy, dummy, dummy, dummy, cnt, None)
        assert rc == api.FWI_ERR_UNSUPPORTED
        assert "column-pair" in api.fwi_last_error()
    other = api.fwi_plan_create(_prob(api, nb=20), api.W2Params())     # another layer width
    plans = (vp * 2)(ok.raw, other.raw)
    assert api._lib.fwi_queue_forward(plans, 2, dummy, dummy, dummy, dummy, cnt, None) == \
        api.FWI_ERR_UNSUPPORTED
    plans = (vp * 5)(*([ok.raw] * 5))
    assert api._lib.fwi_queue_forward(plans, 5, dummy, dummy, dummy, dummy, cnt, None) == \
        api.FWI_ERR_INVALID_ARG


def test_entry_points_reject_misaligned_record_and_workspace_without_a_gpu(api):
    # the record planes and checkpoints move in 16-byte units: a snapshot or
    # workspace pointer off a 16-byte boundary is refused before any CUDA call
    h = api.fwi_plan_create(_prob(api), api.W2Params())
    lib, p, vp = api._lib, h.raw, ctypes.c_void_p
    ok, off = vp(4096), vp(4096 + 8)
    calls = [
        lambda: lib.fwi_forward(p, ok, ok, off, ok, None),
        lambda: lib.fwi_forward(p, ok, ok, ok, off, None),
        lambda: lib.fwi_adjoint_grad(p, ok, ok, off, ok, ok, None),
        lambda: lib.fwi_adjoint_grad(p, ok, ok, ok, ok, off, None),
        lambda: lib.fwi_forward_wait_check(p, ok, ok, off, ok, None),
    ]
    for i, call in enumerate(calls):
        assert call() == api.FWI_ERR_INVALID_ARG, i
        assert "16-byte" in api.fwi_last_error()
    one = (vp * 1)(ok)
    bad = (vp * 1)(off)
    cnt = vp(256)
    plans = (vp * 1)(p)
    # fwi_queue_forward(plans, n, v, d_syn, snapshots, workspace, counter, stream);
    # every call here is refused before a launch
    assert lib.fwi_queue_forward(plans, 1, one, one, bad, one, cnt, None) == api.FWI_ERR_INVALID_ARG
    assert lib.fwi_queue_forward(plans, 1, one, one, one, bad, cnt, None) == api.FWI_ERR_INVALID_ARG
    # fwi_queue_adjoint(plans, n, v, adj_src, snapshots, grad, workspace, counter, stream)
    assert lib.fwi_queue_adjoint(plans, 1, one, one, bad, one, one, cnt, None) == \
        api.FWI_ERR_INVALID_ARG
    assert "16-byte" in api.fwi_last_error()
