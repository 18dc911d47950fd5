"""The FP64 forms' two-pass CFL step: a float screening pass bounds every
cell (double-float pressure, float wave speeds), then FP64 evaluates only the
cells whose float bound is within 1 % of the smallest, or not a positive
finite number.  dt must be the oracle's bit for bit on the exact form and
agree to roundoff on the contracted form, on states built to make the
screen's job hard: the fast-speed discriminant cancelling in every cell
(field along the normal, sound speed = Alfven speed) with the minimum among
thousands of near-equal cells, an exactly uniform state (every cell a
candidate), a single fast cell, densities and pressures spanning nine
decades, and a magnetosphere (inner sphere, dipole) a few steps into its
run."""
import numpy as np
import pytest

from gpu_util import make_gpu, make_oracle
from paper_1607_02214_gb300 import inputs, ppmlr

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_02214_gb300 import build
    build.build()


def periodic(U, n, seed=0):
    edges = [inputs.random_stretched_edges(n[d], seed + d) for d in range(3)]
    return inputs.Problem("screen", edges, GAMMA, inputs.BoundarySpec(powell=1), U)


def degenerate(n=(40, 36, 32), seed=1):
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    rho = np.ones(shape) * (1.0 + 1e-7 * rng.standard_normal(shape))
    Bx = np.full(shape, 1.2)
    p = Bx ** 2 / GAMMA * (1.0 + 1e-7 * rng.standard_normal(shape))      # gamma p = Bx^2: a^2 = b_n^2
    z = np.zeros(shape)
    return periodic(inputs.conserved(rho, (1e-3 * rng.standard_normal(shape), z, z), (Bx, z, z), p, GAMMA), n)


def uniform(n=(24, 20, 18)):
    shape = (n[2], n[1], n[0])
    one = np.ones(shape)
    U = inputs.conserved(one, (0.3 * one, -0.2 * one, 0.1 * one), (0.5 * one, 0.4 * one, -0.3 * one), one, GAMMA)
    edges = [inputs.uniform_axis(k, 0, 1) for k in n]
    return inputs.Problem("uniform", edges, GAMMA, inputs.BoundarySpec(powell=1), U)


def spike(n=(37, 29, 23)):
    pr = periodic(inputs.random_smooth_state(n, 7), n, 7)
    U = pr.U0.copy()
    U[7, 11, 13, 17] *= 30.0                           # one cell with a far higher sound speed
    return inputs.Problem("spike", pr.edges, GAMMA, pr.bc, U)


def wide(n=(33, 27, 25), seed=9):
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    rho = 10.0 ** rng.uniform(-6, 3, shape)
    p = 10.0 ** rng.uniform(-6, 3, shape)
    v = [rng.uniform(-2, 2, shape) for _ in range(3)]
    B = [10.0 ** rng.uniform(-3, 1, shape) * rng.choice([-1, 1], shape) for _ in range(3)]
    return periodic(inputs.conserved(rho, v, B, p, GAMMA), n, seed)


def developing_magnetosphere():
    pr = inputs.magnetosphere(n=(48, 40, 36), h0=1.0)
    o = make_oracle(pr)
    for _ in range(5):
        assert o.step(o.cfl_dt(pr.cfl)) == 0
    return inputs.Problem("magnetosphere_5", pr.edges, pr.gamma, pr.bc, o.get_state(), pr.cfl)


CASES = {"degenerate": degenerate, "uniform": uniform, "spike": spike, "wide": wide,
         "magnetosphere": developing_magnetosphere}


@pytest.mark.parametrize("case", sorted(CASES))
def test_screened_dt_equals_the_oracle(case):
    pr = CASES[case]()
    ref = make_oracle(pr).cfl_dt(0.4)
    assert np.isfinite(ref) and ref > 0
    exact = make_gpu(pr, ppmlr.PPMLR_FP64_EXACT)
    assert exact.cfl_dt(0.4) == ref                                # bit for bit
    assert exact.cfl_dt(0.4) == ref                                # a second call in a row
    fast = make_gpu(pr, ppmlr.PPMLR_FP64)
    assert abs(fast.cfl_dt(0.4) - ref) <= 1e-14 * ref
