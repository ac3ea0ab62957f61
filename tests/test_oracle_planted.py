"""Planted mistakes in the oracle (CPU only): for each, a plausible error in
one step of the oracle makes the pin that guards that step fail.  The
mistakes are patched in for one test only (monkeypatch) and never touch the
device path.  This shows the pins bind: a dropped term, a wrong sign or a
skipped safeguard does not pass unnoticed."""
import importlib

import numpy as np
import pytest

import oracle
from oracle import householder as hh
from oracle import philox, selection

import test_oracle_householder as th
import test_oracle_philox as tp
import test_oracle_rqrcp as tr
import test_oracle_selection as ts

# the module (the package re-exports its function of the same name)
orq = importlib.import_module("oracle.rqrcp")


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_reflector_sign_flip_is_caught(monkeypatch):
    """beta = +sign(alpha)||x|| (a valid reflector, not LAPACK's) changes R."""
    def house_flipped(x):
        x = np.asarray(x, dtype=np.float64)
        alpha, tail = x[0], x[1:]
        xnorm = np.sqrt(np.dot(tail, tail)) if tail.size else 0.0
        v = np.zeros_like(x)
        v[0] = 1.0
        if xnorm == 0.0:
            return v, 0.0, alpha
        beta = np.copysign(np.hypot(alpha, xnorm), alpha if alpha != 0.0 else 1.0)
        v[1:] = tail / (alpha - beta)
        return v, (beta - alpha) / beta, beta
    monkeypatch.setattr(hh, "house", house_flipped)
    _fails(th.test_panel_qr_matches_lapack, 40, 40)


def test_t_factor_sign_error_is_caught(monkeypatch):
    """T[:i, i] = +tau_i T Y^T y_i (sign dropped) no longer reproduces the
    product of the reflectors."""
    def t_factor_wrong(Y, tau):
        b = len(tau)
        T = np.zeros((b, b))
        for i in range(b):
            T[i, i] = tau[i]
            if i > 0:
                T[:i, i] = tau[i] * (T[:i, :i] @ (Y[:, :i].T @ Y[:, i]))
        return T
    monkeypatch.setattr(hh, "t_factor", t_factor_wrong)
    _fails(th.test_t_factor_equals_reflector_product, 20, 6)


def test_block_composition_dropped_coupling_is_caught(monkeypatch):
    """Sec. 5.1 composition without its -T1 Y1^T Y2 T2 block."""
    def compose_wrong(T1, Y1, T2, Y2):
        b1, b2 = T1.shape[0], T2.shape[0]
        T = np.zeros((b1 + b2, b1 + b2))
        T[:b1, :b1] = T1
        T[b1:, b1:] = T2
        return T
    monkeypatch.setattr(hh, "compose_t", compose_wrong)
    _fails(th.test_block_composition)


def test_trailing_update_with_t_instead_of_t_transpose_is_caught(monkeypatch):
    """Applying Q instead of Q^T to the trailing matrix (T for T^T)."""
    def apply_wrong(Y, T, C):
        if C.shape[1] == 0:
            return C
        C -= Y @ (T @ (Y.T @ C))
        return C
    monkeypatch.setattr(orq, "apply_block_transpose", apply_wrong)
    _fails(tr.test_qr_blocked_matches_lapack, 300, 200, 32)


def test_missing_norm_recomputation_is_caught(monkeypatch):
    """Without the exact recomputation of cancelled norms (the xLAQP2
    safeguard) the graded matrix's pivots leave dgeqp3's."""
    monkeypatch.setattr(orq, "TOL3Z", -1.0)
    _fails(tr.test_qrcp_equals_dgeqp3, 120, 120, True)


def test_philox_wrong_round_constant_is_caught(monkeypatch):
    monkeypatch.setattr(philox, "PHILOX_W1", np.uint64(0xBB67AE86))
    ctr, key, out = tp._kat()[0]
    _fails(tp.test_philox_known_answers, ctr, key, out)


def test_selection_wrong_degrees_of_freedom_is_caught(monkeypatch):
    """The sample norms taken chi with l - 1 degrees of freedom."""
    real_chi = selection.stats.chi

    class _Stats:
        @staticmethod
        def chi(df):
            return real_chi(df - 1)
    monkeypatch.setattr(selection, "stats", _Stats)
    _fails(ts.test_two_columns_rayleigh_closed_form, 0.7)


def test_truncation_law_upper_incomplete_gamma_is_caught(monkeypatch):
    """The upper instead of the lower incomplete gamma function in the
    truncated chi-squared expectation (Sec. 3.3)."""
    real = selection.special

    class _Special:
        gammainc = staticmethod(real.gammaincc)
        gamma = staticmethod(real.gamma)
        gammaln = staticmethod(real.gammaln)
    monkeypatch.setattr(selection, "special", _Special)
    _fails(ts.test_truncated_chi2_expectation_is_the_integral, 8, 3.0)


def test_tuxv_misordered_basis_is_caught(monkeypatch):
    """Q formed with its columns reversed: U and V stay orthonormal, but
    U X = A V (and the triangular X) no longer hold (Alg. 7)."""
    real = orq.form_q

    def form_q_reversed(P, tau, ncols):
        return real(P, tau, ncols)[:, ::-1].copy()
    monkeypatch.setattr(orq, "form_q", form_q_reversed)
    _fails(tr.test_tuxv_properties)


def test_rsrqrcp_reused_compression_is_caught(monkeypatch):
    """Alg. 5 that compresses every trailing matrix with the first block's
    Omega instead of a fresh one: valid-looking samples, but not the fresh
    compressions the algorithm defines."""
    def not_fresh(seed, J, ell, trailing):
        return orq.gaussian_block(seed, ell, trailing.shape[0], 1) @ trailing
    monkeypatch.setattr(orq, "_resample", not_fresh)
    _fails(tr.test_rsrqrcp_samples_are_fresh_compressions, 60, 50, 8, 4)


def test_unpatched_pins_pass():
    """The same pins pass on the oracle as written."""
    th.test_panel_qr_matches_lapack(40, 40)
    th.test_t_factor_equals_reflector_product(20, 6)
    th.test_block_composition()
    tr.test_qr_blocked_matches_lapack(300, 200, 32)
    tr.test_qrcp_equals_dgeqp3(120, 120, True)
    ts.test_two_columns_rayleigh_closed_form(0.7)
    ts.test_truncated_chi2_expectation_is_the_integral(8, 3.0)
    tr.test_tuxv_properties()
    tr.test_rsrqrcp_samples_are_fresh_compressions(60, 50, 8, 4)
    ctr, key, out = tp._kat()[0]
    tp.test_philox_known_answers(ctr, key, out)
    assert oracle.rqrcp is not None
