"""The CUDA path's moment transforms on the host (no GPU): m = M f and
f + M^T c of the D3Q19 MRT collision (Eq. 2), written out over shared
partial sums in one-lane (FP32) and two-lane (packed FP32x2) form in
lbm_core.cuh, against the plain matrix products of the d'Humieres moment
basis built here from its polynomials over Eq. 3's velocities
(tests/golden/eq3_d3q19_velocities.txt).  A dropped term, a wrong
coefficient or a swapped pair in the written-out sums fails it."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT, load_golden


def _basis():
    e = load_golden("eq3_d3q19_velocities.txt").astype(int)
    if e.shape[0] == 3:
        e = e.T
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    q = x * x + y * y + z * z
    rows = [np.ones(19), 19 * q - 30, (21 * q * q - 53 * q + 24) / 2, x, (5 * q - 9) * x, y, (5 * q - 9) * y,
            z, (5 * q - 9) * z, 3 * x * x - q, (3 * q - 5) * (3 * x * x - q), y * y - z * z,
            (3 * q - 5) * (y * y - z * z), x * y, y * z, x * z, (y * y - z * z) * x, (z * z - x * x) * y,
            (x * x - y * y) * z]
    return np.array(rows, dtype=np.float64)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tr") / "transforms_check")
    src = os.path.join(ROOT, "tests", "host", "transforms_check.cu")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                        "--expt-relaxed-constexpr", "-o", out, src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_shared_transforms_equal_matrix_products(driver, seed):
    M = _basis()
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, 19).astype(np.float32)
    c = rng.uniform(-1.0, 1.0, 19).astype(np.float32)
    c[[0, 3, 5]] = 0.0   # mass and in-plane momentum are not relaxed
    inp = " ".join("%.9e" % v for v in np.concatenate([f, c]))
    r = subprocess.run([driver], input=inp, capture_output=True, text=True)
    assert r.returncode == 0
    lines = [np.array(list(map(float, ln.split()))) for ln in r.stdout.strip().splitlines()]
    m1, m2x, m2y, b1, b2x, b2y = lines
    f64, c64 = f.astype(np.float64), c.astype(np.float64)
    m_ref = M @ f64
    back_ref = f64 + M.T @ c64
    tol = 2e-5 * np.abs(M).sum(axis=1).max()   # FP32 sums of up to 19 terms of O(1)
    np.testing.assert_allclose(m1, m_ref, atol=tol, rtol=0)
    np.testing.assert_allclose(m2x, m_ref, atol=tol, rtol=0)
    np.testing.assert_allclose(m2y, M @ (-2.0 * f64), atol=2 * tol, rtol=0)
    np.testing.assert_allclose(b1, back_ref, atol=tol, rtol=0)
    np.testing.assert_allclose(b2x, back_ref, atol=tol, rtol=0)
    np.testing.assert_allclose(b2y, -2.0 * f64 + M.T @ (-2.0 * c64), atol=2 * tol, rtol=0)


def test_basis_is_orthogonal():
    """The rows built here are the orthogonal d'Humieres basis (the check
    fails if a polynomial above is mistyped)."""
    M = _basis()
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.linalg.matrix_rank(M) == 19
