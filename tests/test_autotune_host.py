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


def _trial_bytes(prob, steps, fam):
    q = dataclasses.replace(prob, nt=steps, kernels=fam)
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
