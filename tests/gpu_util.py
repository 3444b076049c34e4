"""Helpers of the GPU parity tests: grids, seeded inputs and tolerance bounds."""

import numpy as np
import pytest
import torch

from oracle import fem, mg
from synth import standard_normal

TOL = {"f64": 1e-13, "f32": 4e-6, "bf16": 1.2e-2}
TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def ogrid(n, h, dirichlet):
    return mg.Grid(tuple(n), tuple(h), tuple(dirichlet))


def rounded(a, dt):
    """The array as the GPU will hold it (rounded to the storage type), back in FP64."""
    return torch.as_tensor(a).to(TDT[dt]).to(torch.float64).numpy()


def seeded(shape, seed):
    return standard_normal(seed, int(np.prod(shape))).reshape(shape)


def abs_bound(g, x, k=None):
    """Elementwise bound on sum_j |A_ij x_j| (for rounding-error tolerances)."""
    Ae = np.abs(fem.element_integrals(g.h)["stiff"])
    if k is None:
        return fem.apply_assembled(Ae, np.abs(x))
    ak, ax = np.abs(k), np.abs(x)
    return 0.5 * (fem.apply_assembled(Ae, ak * ax) + ak * fem.apply_assembled(Ae, ax)
                  + ax * fem.apply_assembled(Ae, ak))


def check_close(name, got, ref, rel, scale=None):
    """Max-norm error relative to the reference field's scale (or `scale`), at most `rel`.

    Prints the measured ratio (``PARITY name value``) so that the tolerances can be set from
    the errors actually reached; returns it."""
    scale = max(float(np.abs(ref).max()) if scale is None else float(scale), 1e-300)
    err = float(np.abs(np.asarray(got) - np.asarray(ref)).max()) / scale
    print(f"PARITY {name} {err:.3e} (tol {rel:.1e})")
    assert err <= rel, f"{name}: max rel err {err:.3e} > {rel:.1e}"
    return err
