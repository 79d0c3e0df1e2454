"""Pins of the oracle's IMM constants by the conditions they are chosen to meet.

IMM (Tang, Shi, Xiao, SIGMOD 2015; the algorithm of Sec. II-E, Alg. 2)
picks its two sample-size constants so that two concentration bounds hold
with a stated failure probability. The oracle prints closed forms; these
tests do not retype them. They take the oracle's numbers and check that the
bounds they were derived from come out exactly at their targets:

* ell': the whole run fails with probability at most 2 n^-ell' (one share
  for the lower-bound search, one for the final phase), which must equal
  n^-ell at ell = 1 and stay below it for ell > 1.
* lambda' (lower-bound search): in round i, with x_i = n / 2^i and
  theta_i = lambda' / x_i sets, a seed set whose true spread is at most x_i
  has n F_R(S) >= (1 + eps') x_i with probability at most
  exp(-d^2 / (2 mu + 2 d / 3)) (the martingale upper tail) where
  mu = theta_i x_i / n and d = eps' mu. A union bound over the feasible seed
  sets and the log2 n rounds must bring this to n^-ell' exactly.
* lambda* (final phase): theta = lambda* / OPT sets. The lower tail
  exp(-d^2 / (2 mu)) for the optimal seed set at relative error eps1 must be
  1 / (2 n^ell'); the upper tail for any seed set of spread below
  (gamma - eps) OPT at absolute error eps2 OPT / n, bounded as
  exp(-eps2^2 theta OPT / (2 gamma n)), must be 1 / (2 n^ell' N_S) with N_S
  the number of feasible seed sets; and the error budget must be spent
  exactly: gamma eps1 + eps2 = eps, gamma the greedy's approximation ratio.

For IMM, gamma = 1 - 1/e and N_S = C(n, k). Multi-round IM (Sec. IV-H,
T rounds of k seeds) has N_S = C(n, k)^T and the partition-matroid greedy's
gamma = 1/2 (our reading of the constants, which the paper leaves to its
source). ln C(n, k) comes from Python's exact integer binomial.

Each condition is then shown to catch a slip: the oracle's C source is
compiled with one planted mistake (a dropped term, a wrong logarithm, a
missing factor) and the pins must fail on that copy.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

E_INV = math.exp(-1.0)

# (n, k, eps, ell, T): the workloads' sizes (ER n = 2000; R-MAT scale 20 and
# 22; the multi-round workload), plus a few off-grid points.
CASES = [
    (2000, 10, 0.5, 1.0, 1),
    (1 << 20, 50, 0.1, 1.0, 1),
    (1 << 22, 100, 0.05, 1.0, 1),
    (1 << 22, 50, 0.1, 1.0, 1),
    (1 << 22, 100, 0.2, 1.0, 1),
    (1_000_000, 50, 0.05, 1.0, 1),
    (4096, 7, 0.3, 2.0, 1),
    (1 << 22, 10, 0.1, 1.0, 5),
    (2000, 10, 0.5, 1.0, 3),
    (1 << 20, 25, 0.2, 1.5, 2),
]


def _ln_binom_exact(n, k):
    return math.log(math.comb(n, k))


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_constants(c, n, k, eps, ell, T):
    """Returns the relative residuals of every condition for constants c."""
    ln_n = math.log(n)
    ln_ns = T * _ln_binom_exact(n, k)               # ln of the number of feasible seed sets
    gamma = (1.0 - E_INV) if T == 1 else 0.5
    ellp, epsp, lam1, lam2 = c["ell_prime"], c["eps_prime"], c["lambda_prime"], c["lambda_star"]
    res = {}

    # ell': total failure 2 n^-ell' against the target n^-ell, in logs; equality at ell = 1.
    res["ell_prime"] = _rel(math.log(2.0) - ellp * ln_n, -ell * ln_n - (ell - 1.0) * math.log(2.0))

    # eps': Alg. 2 tests n F_R(S) >= (1 + sqrt(2) eps) x.
    res["eps_prime"] = _rel(epsp * epsp, 2.0 * eps * eps)

    # lambda': the martingale upper tail at the worst admissible spread x_i,
    # union over the feasible seed sets and the rounds, equals n^-ell'.
    worst = 0.0
    for i in (1, 2, max(1, n.bit_length() - 2)):
        x = n / 2.0 ** i
        theta_i = lam1 / x
        mu = theta_i * x / n
        d = epsp * mu
        log_tail = -(d * d) / (2.0 * mu + 2.0 * d / 3.0)
        log_union = log_tail + ln_ns + math.log(math.log2(n))
        worst = max(worst, _rel(log_union, -ellp * ln_n))
    res["lambda_prime"] = worst

    # lambda*: solve each tail bound for the error it allows at theta * OPT = lambda*
    opt = n / 7.0                                   # any OPT: only theta * OPT enters
    theta = lam2 / opt
    log_d1 = -(math.log(2.0) + ellp * ln_n)         # delta1 = 1 / (2 n^ell')
    log_d2 = log_d1 - ln_ns                         # delta2 = delta1 / N_S
    mu = theta * opt / n
    eps1 = math.sqrt(-log_d1 * 2.0 * mu) / mu       # exp(-(eps1 mu)^2 / (2 mu)) = delta1
    eps2 = math.sqrt(-log_d2 * 2.0 * gamma * n / (theta * opt))   # exp(-eps2^2 theta OPT / (2 gamma n)) = delta2
    res["budget"] = _rel(gamma * eps1 + eps2, eps)
    # the simplified upper tail is a valid bound: with spread p = (gamma - eps) OPT / n and
    # deviation eps2 theta OPT / n, 2 theta p + 2 dev / 3 <= 2 gamma theta OPT / n
    p = (gamma - eps) * opt / n
    dev = eps2 * theta * opt / n
    res["upper_tail_valid"] = 0.0 if 2 * theta * p + 2 * dev / 3 <= 2 * gamma * theta * opt / n * (1 + 1e-15) else 1.0
    return res


TOL = 1e-12


@pytest.mark.parametrize("n,k,eps,ell,T", CASES)
def test_constants_meet_their_bounds(oracle_mod, n, k, eps, ell, T):
    c = oracle_mod.mrim_constants(n, k, T, eps, ell)
    if T == 1:
        assert c == oracle_mod.imm_constants(n, k, eps, ell)
    res = check_constants(c, n, k, eps, ell, T)
    bad = {key: v for key, v in res.items() if v > TOL}
    assert not bad, bad


def test_ell_prime_is_tight_only_at_ell_one(oracle_mod):
    n = 1 << 22
    for ell in (1.0, 1.5, 3.0):
        c = oracle_mod.imm_constants(n, 50, 0.1, ell)
        fail = math.log(2.0) - c["ell_prime"] * math.log(n)       # ln of 2 n^-ell'
        target = -ell * math.log(n)
        if ell == 1.0:
            assert _rel(fail, target) < TOL
        else:
            assert fail < target


# ---------------------------------------------------------------------------
# Planted slips: each one, compiled into a copy of the oracle, fails a pin.
# ---------------------------------------------------------------------------
_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gim_oracle.c")

SLIPS = {
    # ln ln n instead of ln log2 n in lambda'
    "lnln_in_lambda_prime": ("log(log2((double)n))", "log(log((double)n))"),
    # (1 - 1/e) dropped from beta
    "beta_without_gamma": ("sqrt(gamma * (lnC + ellp * ln_n + log(2.0)))", "sqrt((lnC + ellp * ln_n + log(2.0)))"),
    # ln 2 dropped from alpha
    "alpha_without_ln2": ("sqrt(ellp * ln_n + log(2.0))", "sqrt(ellp * ln_n)"),
    # gamma alpha + beta written as alpha + beta
    "alpha_without_gamma": ("gamma * alpha + beta", "alpha + beta"),
    # the ell adjustment without the 1 / ln n
    "ell_prime_slip": ("ell * (1.0 + log(2.0) / ln_n)", "ell * (1.0 + log(2.0))"),
    # the T rounds' seed sets counted once
    "multi_round_lnC_once": ("(double)T * orc_log_binom(n, k)", "orc_log_binom(n, k)"),
    # (2 + 2 eps'/3) written as (2 + eps'/3)
    "martingale_factor": ("(2.0 + 2.0 * epsp / 3.0)", "(2.0 + epsp / 3.0)"),
}


def _planted(tmp_path, name):
    old, new = SLIPS[name]
    src = open(_SRC).read()
    assert src.count(old) == 1, (name, src.count(old))
    path = tmp_path / f"slip_{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"slip_{name}.so"
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", str(path), "-o", str(so),
                    "-lm"], check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_mrim_constants.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                       ctypes.c_double, np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")]
    lib.orc_mrim_constants.restype = None

    def consts(n, k, T, eps, ell):
        out = np.zeros(5, np.float64)
        lib.orc_mrim_constants(n, k, T, eps, ell, out)
        return dict(ell_prime=out[0], eps_prime=out[1], lambda_prime=out[2], lambda_star=out[3], i_max=int(out[4]))
    return consts


@pytest.mark.parametrize("name", sorted(SLIPS))
def test_planted_slip_fails_a_pin(tmp_path, name):
    consts = _planted(tmp_path, name)
    caught = False
    for n, k, eps, ell, T in CASES:
        res = check_constants(consts(n, k, T, eps, ell), n, k, eps, ell, T)
        if any(v > TOL for v in res.values()):
            caught = True
            break
    assert caught, name
