"""The evaluation kernel's erfc (Eq. 3 needs 12 per pair) is a fitted
rational form with constants in dsc_erfc_coeffs.h and dsc_kernels.cu.  This
pins those constants on the CPU against scipy's erfc, independently of the
oracle: the fitted form's error in FP64, the same form evaluated with FP32
roundings (Horner in FMA steps, as the kernel does), and the scaling
constants that turn u into v = u sqrt(log2 e)."""
import math
import os
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")
CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0908_4417_gb300", "csrc")


def header():
    src = open(os.path.join(CSRC, "dsc_erfc_coeffs.h")).read()
    p = float(re.search(r"kErfcP = ([-0-9.e+]+)f", src).group(1))
    n = int(re.search(r"kErfcN = (\d+)", src).group(1))
    def arr(name, pairs):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        vals = [float(v) for v in re.findall(r"([-0-9.]+e[-+]\d+)f", body)]
        return np.array(vals).reshape(-1, 2) if pairs else np.array(vals)
    return p, n, arr("kErfcC", False), arr("kErfcC2", True), arr("kErfcC2n", True)


def test_packed_tables_repeat_the_scalar_coefficients():
    p, n, c, c2, c2n = header()
    assert len(c) == n + 1 and c2.shape == (n + 1, 2) and c2n.shape == (n + 1, 2)
    assert np.array_equal(c2[:, 0], c) and np.array_equal(c2[:, 1], c)
    assert np.array_equal(c2n[:, 0], -c) and np.array_equal(c2n[:, 1], -c)


def test_fitted_form_error_fp64_and_fp32():
    p, n, c, _, _ = header()
    x = np.linspace(0.0, 9.5, 400001)
    t = 1.0 / (1.0 + p * x)
    P = np.polyval(c[::-1], t)
    rel64 = np.abs(t * P * np.exp(-x * x) - special.erfc(x)) / special.erfc(x)
    assert rel64.max() < 2e-7
    # FP32: t from a correctly rounded reciprocal, Horner with one rounding per FMA
    f = np.float32
    xf = x.astype(f)
    tf = (1.0 / (f(p) * xf.astype(np.float64) + 1.0).astype(f).astype(np.float64)).astype(f)
    acc = np.full_like(tf, f(c[-1]))
    for ck in c[-2::-1]:
        acc = (acc.astype(np.float64) * tf + f(ck)).astype(f)
    tp = (tf.astype(np.float64) * acc).astype(f).astype(np.float64)
    ref = special.erfcx(xf.astype(np.float64))
    assert (np.abs(tp - ref) / ref).max() < 5e-7


def test_scaling_constants():
    src = open(os.path.join(CSRC, "dsc_kernels.cu")).read()
    inv_sqrt_l = float(re.search(r"kInvSqrtL = ([0-9.]+)f", src).group(1))
    K = {int(m.group(1)): float(m.group(2)) for m in
         re.finditer(r"struct Prof<(\d)> \{ static constexpr float K = ([0-9.]+)f", src)}
    sqrt_half_l = K[0]
    # the other profiles' scales: Laplace s = c3/sqrt 2, logistic s = c3 sqrt 3/pi, both in log2 units
    assert abs(K[1] - math.sqrt(2.0) / math.log(2.0)) < 1e-15
    assert abs(K[2] - math.pi / math.sqrt(3.0) / math.log(2.0)) < 1e-15
    log2e = 1.0 / math.log(2.0)
    assert abs(inv_sqrt_l - 1.0 / math.sqrt(log2e)) < 1e-15
    assert abs(sqrt_half_l - math.sqrt(log2e / 2.0)) < 1e-15
    # exp(-u^2) == 2^(-v^2) with v = u sqrt(log2 e); erf argument (h -/+ x)/(sqrt(2) sigma) -> v scale
    u = 1.7
    assert abs(math.exp(-u * u) - 2.0 ** (-(u * math.sqrt(log2e)) ** 2)) < 1e-15
    assert abs(sqrt_half_l - math.sqrt(log2e) / math.sqrt(2.0)) < 1e-15


def test_erf_pair_identity():
    """erf(u1) + erf(u2) = erfc(-u1) - erfc(u2), and erfc(-x) = 2 - erfc(x):
    the two forms the kernel selects by the sign of -u1."""
    for h, x, s in ((2.5, 0.3, 1.2), (2.5, 7.0, 0.8), (0.1, 3.0, 2.0), (1.0, 1.0, 1.0)):
        u1, u2 = (h - x) / s, (h + x) / s
        lhs = math.erf(u1) + math.erf(u2)
        assert abs(lhs - (special.erfc(-u1) - special.erfc(u2))) < 1e-14
        if -u1 < 0:
            assert abs(lhs - (2.0 - special.erfc(u1) - special.erfc(u2))) < 1e-14
