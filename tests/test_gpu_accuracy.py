"""Accuracy of each storage format on the 384^3 body-force channel (the paper's
verification set-up, Sec. 2.1, at F = 1e-7 for 5000 steps).

The oracle runs the 2 x 384 x 2 column: a channel run is bitwise independent
of x and z (pinned in test_oracle_pins), so the column is the 3-D reference.
Errors of the mean velocity profile u_x(y) are reported against the oracle
and against the analytic start-up series evaluated at t + 1/2. Set
LBM_ACCURACY_REPORT=<path> to write them as JSON.
"""
import json
import os

import numpy as np
import pytest

from paper_1711_11468_gb300 import inputs

pytestmark = pytest.mark.gpu

# Max-relative error of the profile against the FP64 oracle, per storage format:
# (lower, upper) bounds around the values measured on GB300, with the outcome each
# records against the workload's FP32 target of 1e-5.
#  - FP64 and FP64 storage with the double-float collision: about 1e-10, the random
#    round-off walk of a profile (u ~ 5e-4) built from PDFs of size ~0.1.
#  - FP32 storage MISSES the target (measured 4.2e-5): the 1e-8-per-step force
#    increment is rounded against values near 1e-4, with FP32 collision arithmetic.
#  - FP32 storage with the double-float collision MEETS it (measured 3.3e-6): the
#    stored values are rounded once per step, without the correlated rounding of
#    FP32 arithmetic.
#  - FP16 storage STAGNATES (measured 1.0): the increments fall below half an FP16
#    spacing, so the profile stays at rest; the lower bound asserts the stagnation.
#  - Scaled FP16 storage with stochastic rounding keeps the increments on average
#    (measured 4.4e-5): the noise of the random rounding averaged over the 384^2
#    cells of a plane, the level of FP32 storage, at half its bytes.
BOUNDS = {0: (0.0, 1e-9), 3: (0.0, 1e-9), 1: (1e-5, 8e-5), 4: (0.0, 1e-5), 2: (0.9, 1.1), 5: (0.0, 8e-5)}
OUTCOME = {0: "round-off", 3: "round-off", 1: "misses 1e-5", 4: "meets 1e-5", 2: "stagnates",
           5: "FP32 level"}


def series(y, t, F, nu, a, b, nterms=4001):
    L = b - a
    s = F / (2 * nu) * (y - a) * (b - y)
    for n in range(1, nterms, 2):
        s = s - 4 * F * L * L / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * (y - a) / L) \
            * np.exp(-nu * n * n * np.pi ** 2 * t / L ** 2)
    return s


@pytest.fixture(scope="module")
def reference(orc):
    c = inputs.CHANNEL_384
    ny = c["dims"][1]
    dims = (2, ny, 2)
    fl = inputs.channel_flags(*dims)
    f = orc.run(dims, fl, c["omega"], orc.omega_minus(c["omega"], c["Lambda"]), c["force"],
                orc.init_equilibrium(dims, fl), c["steps"])
    _, u = orc.macroscopic(dims, fl, c["force"], f)
    prof = u[0].reshape(2, ny, 2)[0, :, 0]
    nu = (1.0 / c["omega"] - 0.5) / 3.0
    ana = series(np.arange(ny, dtype=float), c["steps"] + 0.5, c["force"][0], nu, 0.5, ny - 1.5)
    return prof, ana


REPORT = {}


@pytest.mark.parametrize("prec", [1, 4, 2, 5, 3, 0])
def test_channel384_profile_error(lbm, reference, prec):
    import torch
    c = inputs.CHANNEL_384
    dims = c["dims"]
    ny = dims[1]
    h = lbm.lbm_create_lattice(lbm.make_desc(dims, prec, lbm.LBM_DIRECT, lbm.LBM_AA_INPLACE, (1, 0, 1)),
                               torch.cuda.current_stream())
    try:
        lbm.lbm_set_geometry(h, 0, inputs.channel_flags(*dims))
        lbm.lbm_set_params(h, 0, c["omega"], c["Lambda"], c["force"])
        lbm.lbm_init_equilibrium(h, 0)
        lbm.lbm_step(h, c["steps"])
        prof = lbm.lbm_read_profile(h, 0, 1, 0)
        mass = lbm.lbm_read_moments(h, 0)[0]
    finally:
        lbm.lbm_destroy(h)
    ref, ana = reference
    m = slice(1, ny - 1)
    scale = np.abs(ref[m]).max()
    err = {
        "max_rel_vs_oracle": float(np.abs(prof[m] - ref[m]).max() / scale),
        "l2_rel_vs_oracle": float(np.linalg.norm(prof[m] - ref[m]) / np.linalg.norm(ref[m])),
        "max_rel_vs_analytic": float(np.abs(prof[m] - ana[m]).max() / np.abs(ana[m]).max()),
        "oracle_max_rel_vs_analytic": float(np.abs(ref[m] - ana[m]).max() / np.abs(ana[m]).max()),
        "mass_rel_drift": float(abs(mass - np.prod(dims)) / np.prod(dims)),
    }
    name = {0: "f64", 1: "f32_shifted", 2: "f16_shifted", 3: "f64_double_float",
            4: "f32_shifted_double_float", 5: "f16_shifted_stochastic"}[prec]
    REPORT[name] = err
    path = os.environ.get("LBM_ACCURACY_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump({"workload": "channel 384^3, F=1e-7, omega=1, Lambda=3/16, 5000 steps, AA",
                       "errors": REPORT}, fh, indent=1)
    assert np.all(np.isfinite(prof))
    lo, hi = BOUNDS[prec]
    assert lo <= err["max_rel_vs_oracle"] <= hi, (OUTCOME[prec], err)
