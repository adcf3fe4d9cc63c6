"""Host-side checks of the kernel-family autotuner's sizing and argument
validation (no GPU): the scratch it asks for covers every family's trial
plan (workspace + snapshots + data + gradient, 256-byte aligned pieces)."""
import dataclasses

import pytest

from paper_2603_16393_gb300 import api



def _prob(**kw):
    base = dict(nz=70, nx=70, nb=40, nt=1000, dz=10.0, dx=10.0, dt=1e-3,
                src_iz=(0,) * 5, src_ix=(0, 17, 34, 52, 69), rec_iz=(0,) * 70,
                rec_ix=tuple(range(70)), v_max=4500.0, batch=3)
    base.update(kw)
    return api.Problem(**base)


def _up(n):
    return -(-n // 256) * 256


SHAPES = {api.KERNELS_RESIDENT: (api.SHAPE_RESIDENT_PAIRS, api.SHAPE_RESIDENT_COLUMNS),
          api.KERNELS_TILED: (api.SHAPE_TILED_ROWS8, api.SHAPE_TILED_ROWS4,
                              api.SHAPE_TILED_QUADS),
          api.KERNELS_CLUSTER: (api.SHAPE_CLUSTER_PAIRS, api.SHAPE_CLUSTER_RS13,
                            api.SHAPE_CLUSTER_RS19),
          api.KERNELS_CPML: (api.SHAPE_DEFAULT,)}


def _trial_bytes(prob, steps, fam):
    """The largest trial buffer over the family's shapes (None: the family
    cannot run the problem)."""
    sizes = [b for b in (_shape_bytes(prob, steps, fam, sh) for sh in SHAPES[fam]) if b]
    return max(sizes) if sizes else None


def _shape_bytes(prob, steps, fam, shape):
    q = dataclasses.replace(prob, nt=steps, kernels=fam, shape=shape)
    try:
        h = api.fwi_plan_create(q, api.W2Params())
    except api.FwiError as e:
        assert e.code == 3
        return None
    ws, _, snap = api.fwi_plan_sizes(h)
    data = q.batch * q.ns * q.nr * steps * 4
    grad = q.batch * q.nz * q.nx * 4
    return _up(ws) + _up(snap) + _up(data) + _up(grad)


@pytest.mark.parametrize("kw,families", [
    (dict(), 3),                                   # 110 x 150 cells: all three families
    (dict(nz=100, nx=140, nb=20, src_ix=(0, 70, 139), src_iz=(0,) * 3,
          rec_iz=(0,) * 140, rec_ix=tuple(range(140))), 2),   # beyond one CTA: tiled, cluster
    (dict(space_order=8), 1),                      # 8th order: tiled only
    (dict(absorber=1), 1),                         # CPML absorber: its own kernels only
])
def test_scratch_covers_every_family(kw, families):
    prob = _prob(**kw)
    steps = 48              # the trials run 48 and 96 steps: the scratch fits the longer
    need = [_trial_bytes(prob, 2 * steps, f) for f in (api.KERNELS_RESIDENT, api.KERNELS_TILED,
                                                       api.KERNELS_CLUSTER, api.KERNELS_CPML)]
    ok = [n for n in need if n is not None]
    assert len(ok) == families
    assert api.fwi_autotune_scratch_bytes(prob, api.W2Params(), steps) == max(ok)
    # a trial of more than half the steps is capped at nt
    short = dataclasses.replace(prob, nt=60)
    cap = [_trial_bytes(short, 60, f) for f in (api.KERNELS_RESIDENT, api.KERNELS_TILED,
                                                api.KERNELS_CLUSTER, api.KERNELS_CPML)]
    assert api.fwi_autotune_scratch_bytes(short, api.W2Params(), 40) == max(
        n for n in cap if n is not None)


def test_autotune_rejects_bad_arguments():
    prob = _prob()
    for steps in (1, 1001):
        with pytest.raises(api.FwiError) as e:
            api.fwi_autotune_scratch_bytes(prob, api.W2Params(), steps)
        assert e.value.code == 1
    with pytest.raises(api.FwiError) as e:          # the problem itself is unstable
        api.fwi_autotune_scratch_bytes(_prob(v_max=9000.0), api.W2Params(), 32)
    assert e.value.code == 2


def test_shapes_belong_to_their_family():
    prob = _prob()
    for fam, shapes in SHAPES.items():
        if fam == api.KERNELS_CPML:
            continue
        for sh in shapes:
            api.fwi_plan_create(dataclasses.replace(prob, kernels=fam, shape=sh), api.W2Params())
        others = [x for f, ss in SHAPES.items() if f != fam for x in ss if x]
        for sh in others:
            with pytest.raises(api.FwiError) as e:
                api.fwi_plan_create(dataclasses.replace(prob, kernels=fam, shape=sh),
                                    api.W2Params())
            assert e.value.code == 3 and "shape" in str(e.value)
    with pytest.raises(api.FwiError) as e:
        api.fwi_plan_create(dataclasses.replace(prob, shape=9), api.W2Params())
    assert e.value.code == 1
    # an odd padded width has no column pairs
    odd = _prob(nx=69, src_ix=(0, 17, 34, 51, 68), rec_ix=tuple(range(69)), rec_iz=(0,) * 69)
    with pytest.raises(api.FwiError):
        api.fwi_plan_create(dataclasses.replace(odd, shape=api.SHAPE_RESIDENT_PAIRS),
                            api.W2Params())
    api.fwi_plan_create(dataclasses.replace(odd, shape=api.SHAPE_RESIDENT_COLUMNS), api.W2Params())
    # ... nor cluster column pairs: the single-column strips take the grid
    big = _prob(nz=200, nx=201, src_ix=(0, 50, 100, 150, 200), rec_ix=tuple(range(201)),
                rec_iz=(0,) * 201)
    with pytest.raises(api.FwiError):
        api.fwi_plan_create(dataclasses.replace(big, kernels=api.KERNELS_CLUSTER,
                                                shape=api.SHAPE_CLUSTER_PAIRS), api.W2Params())
    p = api.fwi_plan_create(dataclasses.replace(big, kernels=api.KERNELS_CLUSTER),
                            api.W2Params())
    assert api.fwi_plan_kernels(p) == api.KERNELS_CLUSTER
