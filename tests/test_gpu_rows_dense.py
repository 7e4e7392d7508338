"""GPU parity of the FP64 Gibbs operator on dense costs (the rows kernel with
an FP32 prefilter, Sec. 4.3's log-domain operator) against the oracle's
apply_K_log, on shapes that take each of its branches:

- rows of nin % 4 == 0 that fit (four rows and the line in 96 KB) are staged in
  shared memory before the kernel waits for its predecessor; other rows are
  read from global memory, with the line in shared memory up to 12288 columns
  (above 48 KB per block with the static lists: the opt-in size) and in global
  memory beyond;
- small eps (most terms below e^-746, a few survivors per row), large eps
  (every term survives: full 32-term batches per warp), a potential that makes
  the row maximum move along the whole row, +inf costs (WF cut locus), and a
  solve over 10001 rows against 64 (the other pass: 64 rows of 10001 columns).

The bar is the FP64 tolerance of every parity test: 1e-10 relative to
max(1, |reference|_inf)."""
import numpy as np
import pytest

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

from test_gpu_parity import TOL, T, rel_err, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def dense_case(n, m, seed, cost="sqdist", cut=0.2):
    g = synth.rng(seed)
    x = np.sort(g.uniform(0, 1, size=n))
    y = np.sort(g.uniform(0, 1, size=m))
    C = O.sqdist(x, y) if cost == "sqdist" else O.wf_cost(x[:, None], y[:, None], cut)
    return x, y, C


def check(C, W, w, eps, transpose):
    want = O.apply_K_log(O.Geometry("dense", C=C), W, np.log(w), eps, transpose=transpose)
    got = to_np(U.gibbs_log(U.Geometry.dense(T(C, U.F64)), T(W, U.F64), T(w, U.F64), eps, transpose, U.F64))
    assert np.array_equal(np.isneginf(got), np.isneginf(want))
    assert rel_err(got, want) <= TOL[U.F64]


@pytest.mark.parametrize("n,m,eps,transpose", [
    (97, 132, 1e-2, False),    # staged rows, a ragged last CTA
    (97, 132, 1e-2, True),     # nin = 97: rows from global memory, line in shared memory
    (600, 1024, 1e-6, False),  # few survivors per row
    (33, 8192, 5e-2, False),   # thousands of survivors per row: full batches
    (40, 12300, 5e-2, False),  # rows and line from global memory
    (10001, 16, 1e-2, False),  # many short rows
])
def test_dense_rows_parity(n, m, eps, transpose):
    x, y, C = dense_case(n, m, 3 + n)
    g = synth.rng(n + m)
    nin = n if transpose else m
    W = g.normal(size=nin) * 0.05
    W[7::23] = -np.inf
    w = g.uniform(0.5, 1.5, size=nin) / nin
    check(C, W, w, eps, transpose)


@pytest.mark.parametrize("eps", [1e-8, 1e-4])
def test_dense_rows_running_maximum_moves_along_the_row(eps):
    """W_j = 2 y_j: for the first rows t_j = (2 y_j - (x_i - y_j)^2)/eps grows
    along the whole row, so every block that the first sweep marks early is
    later far below the row maximum, and the survivors sit in the last block."""
    x, y, C = dense_case(256, 2048, 17)
    check(C, 2.0 * y, np.full(2048, 1.0 / 2048), eps, False)
    # and a decreasing ramp: the maximum in the first block, survivors there only
    check(C, -2.0 * y, np.full(2048, 1.0 / 2048), eps, False)


@pytest.mark.parametrize("eps", [1e-8, 1e-3])
def test_dense_rows_wf_cost_with_cut_locus(eps):
    """The WF cost is +inf beyond the cut locus: those terms vanish; W of the
    paper's scale (potentials of order 1 at eps = 1e-8)."""
    x, y, C = dense_case(1200, 1200, 29, cost="wf", cut=0.2)
    assert np.isposinf(C).any()
    g = synth.rng(31)
    W = g.uniform(-1.0, 0.0, size=1200)
    W[::97] = -np.inf
    check(C, W, np.full(1200, 1.0 / 1200), eps, False)
    check(C, W, np.full(1200, 1.0 / 1200), eps, True)


def test_dense_rows_all_inputs_zero():
    """b = 0 everywhere (W = -inf): every output is an empty sum (-inf)."""
    x, y, C = dense_case(64, 256, 5)
    W = np.full(256, -np.inf)
    got = to_np(U.gibbs_log(U.Geometry.dense(T(C, U.F64)), T(W, U.F64), T(np.full(256, 1 / 256), U.F64), 1e-2,
                            False, U.F64))
    assert np.all(np.isneginf(got))


def test_dense_solve_long_and_short_rows_matches_oracle():
    """A KL solve on a 10001 x 64 cost: 10001 short staged rows one way, 64
    rows of 10001 columns (line in opt-in shared memory) the other, with the
    violation accumulated over every CTA."""
    x, y, C = dense_case(10001, 64, 41)
    dx, dy = np.full(10001, 1.0 / 10001), np.full(64, 1.0 / 64)
    g = synth.rng(43)
    p, q = g.uniform(0.5, 1.5, 10001), g.uniform(0.5, 1.5, 64)
    r = O.solve_log(O.Geometry("dense", C=C), dx, dy, p, q, O.KL(0.5), O.KL(0.5), 1e-2, max_iter=30, stages=0)
    Ug, Vg, info = U.solve(U.Geometry.dense(T(C, U.F64)), T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64),
                           U.KL(0.5), U.KL(0.5), 1e-2, precision=U.F64, max_iter=30, eps_stages=0, check_every=1)
    assert info["status"] == "UOT_OK" and info["total_iters"] == 30
    # the violation accumulated over every CTA is the oracle's
    assert abs(info["marg_err"] - r["err"]) <= 1e-8 * max(1.0, r["err"])
    assert rel_err(to_np(Ug), r["U"]) <= TOL[U.F64]
    assert rel_err(to_np(Vg), r["V"]) <= TOL[U.F64]
