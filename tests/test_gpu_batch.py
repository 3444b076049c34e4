"""GPU parity of the batched pressure solve (one launch per cycle step over all instances).

* FP64 storage, one cycle per outer iteration: after k outer iterations every instance equals the
  oracle's k sawtooth cycles to 1e-12 (the defect-correction form of the same iteration);
* FP32 / BF16 storage: every instance reaches its own FP64 solution (oracle CG to 1e-14) to 1e-8;
  instances converge independently (per-instance iteration counts and latencies).
Instances have uneven sizes (17, 25, 33 and 9 x 17 x 33 nodes) and mixed face conditions.
"""

import numpy as np
import pytest
import torch

from oracle import direct, fem, mg
from synth import standard_normal
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

SPECS = [
    ((17, 17, 17), (False,) * 5 + (True,)),
    ((33, 33, 33), (True,) * 6),
    ((25, 25, 25), (False,) * 5 + (True,)),
    ((9, 17, 33), (False,) * 5 + (True,)),
    ((33, 17, 17), (True,) * 6),
]


def _setup(seed0=0):
    from paper_2401_06755_gb300 import nn4
    gs, Gs, bs = [], [], []
    for i, (n, bc) in enumerate(SPECS):
        h = 1.0 / 32
        g = mg.Grid(n, (h,) * 3, bc)
        G = nn4.Grid(n, (h,) * 3, tuple(nn4.DIRICHLET if d else nn4.NATURAL for d in bc))
        b = fem.lumped_mass(g.shape, g.h) * standard_normal(seed0 + i, int(np.prod(g.shape))).reshape(g.shape)
        b[mg.dirichlet_mask(g)] = 0.0
        gs.append(g)
        Gs.append(G)
        bs.append(b)
    return nn4, gs, Gs, bs


def test_batched_fp64_matches_oracle_cycles():
    need_gpu()
    nn4, gs, Gs, bs = _setup()
    batch = nn4.Batch(Gs, inner=nn4.F64, inner_cycles=1)
    B = [nn4.to_field(b, G) for b, G in zip(bs, Gs)]
    X = [nn4.field(G) for G in Gs]
    k = 6
    code, infos, lat = batch.solve(B, X, rtol=0.0, max_iters=k)
    for g, G, b, x, info in zip(gs, Gs, bs, X, infos):
        xo, _ = mg.pressure_solve(g, b, fixed_cycles=k)
        xg = nn4.nodes(x, G).cpu().numpy()
        assert info["iterations"] == k
        assert np.linalg.norm(xg - xo) <= 1e-12 * np.linalg.norm(xo)


@pytest.mark.parametrize("inner,cycles", [("f32", 2), ("f32", 4), ("bf16", 2)])
def test_batched_mixed_reaches_fp64_solutions(inner, cycles):
    need_gpu()
    nn4, gs, Gs, bs = _setup(10)
    batch = nn4.Batch(Gs, inner=nn4.F32 if inner == "f32" else nn4.BF16, inner_cycles=cycles)
    B = [nn4.to_field(b, G) for b, G in zip(bs, Gs)]
    X = [nn4.field(G) for G in Gs]
    code, infos, lat = batch.solve(B, X, rtol=1e-10, max_iters=100)
    assert code == nn4.OK
    for g, G, b, x, info, t in zip(gs, Gs, bs, X, infos, lat):
        xref = direct.solve_cg(g, b, rtol=1e-14)
        xg = nn4.nodes(x, G).cpu().numpy()
        assert info["rel_res"] <= 1e-10
        assert np.linalg.norm(xg - xref) <= 1e-8 * np.linalg.norm(xref)
        assert t > 0.0
    # instances stop independently: their iteration counts differ
    its = [i["iterations"] for i in infos]
    assert max(its) > min(its)


@pytest.mark.parametrize("shape", [1, 2, 3])
def test_batched_forced_tile_shape_matches_oracle_cycles(shape):
    """Every compiled tile shape of the batched Jacobi launch (forced through pass_shape) gives the
    oracle's sawtooth cycles to 1e-12 per instance after six FP64 iterations."""
    need_gpu()
    nn4, gs, Gs, bs = _setup()
    batch = nn4.Batch(Gs, inner=nn4.F64, inner_cycles=1, pass_shape=shape)
    assert all(e["shape"] == shape for e in batch.query())
    B = [nn4.to_field(b, G) for b, G in zip(bs, Gs)]
    X = [nn4.field(G) for G in Gs]
    k = 6
    batch.solve(B, X, rtol=0.0, max_iters=k)
    for g, G, b, x in zip(gs, Gs, bs, X):
        xo, _ = mg.pressure_solve(g, b, fixed_cycles=k)
        xg = nn4.nodes(x, G).cpu().numpy()
        assert np.linalg.norm(xg - xo) <= 1e-12 * np.linalg.norm(xo)


def test_batched_autotuner_reports_its_choice():
    """With autotuning on, every level step's Jacobi launch was timed at creation; the choice is a
    compiled shape and z cap, and level 0 covers the finest nodes of every instance."""
    need_gpu()
    nn4, gs, Gs, bs = _setup()
    batch = nn4.Batch(Gs, inner=nn4.F32, inner_cycles=2)
    q = batch.query()
    assert q and q[0]["nodes"] == sum(int(np.prod(G.n)) for G in Gs)
    for e in q:
        if e["items"] == 0:
            continue
        assert 0 <= e["shape"] < 4 and e["zmax"] in (16, 32, 64) and e["jacobi_us"] > 0.0
