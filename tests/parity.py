"""Shared helpers for the GPU parity tests (test code; imports the oracle).

Tolerances.  The RHS of a variable is a sum of flux-divergence terms of
magnitude about J |Dt| |F| that cancel to a much smaller result (by a
factor up to ~1e5 for the auxiliary equations, whose result is
(grad u - q)/T).  Floating-point error is proportional to the terms, not
to the result, so the parity bound for variable v is

    || R_gpu,v - R_oracle,v ||_2  <=  tol * || B_v ||_2,
    B_v = sum_a J_a sum_k |Dt_ik| |F_a,v,k|  +  |S_v|,

with tol = 1e-12 (FP64) and 2e-5 (FP32), the oracle evaluated in FP64 on
the identical (already rounded) input values.  Where the result does not
cancel, the plain relative bound || dR_v || <= tol || R_oracle,v || must
hold as well, for every variable whose || R_v || / || B_v || is at least
CANCEL_MIN[precision].  That threshold follows from the arithmetic: any
evaluation in a precision with unit roundoff u carries an error of about
k u || B_v || (k a small count of roundings; measured k ~ 1-2 here), so the
plain bound tol || R_v || is attainable only where || R_v || / || B_v || >=
k u / tol.  With k = 8: FP32 (u = 2^-24) 2.4e-2, FP64 (u = 2^-53) 1e-3
(k u / tol ~ 1e-3 too).  Rows whose result cancels further (the auxiliary
rows' (grad u - q)/T by up to 1e5; P and V of nearly divergence-free or
steady fields) are held to the scaled bound.

With ACMHD_PARITY_LOG=<path> set, every check appends one JSON line (label,
precision, per-variable scaled and plain errors, |R|/|B|) to that file.
"""
import json
import os

import numpy as np

from oracle import acmhd, fr
from oracle.ops1d import Ops1D
from paper_2107_14027_gb300 import workloads as W

# 65: FR_DF64 (FP64 storage, double-float arithmetic, unit roundoff ~2^-48)
TOL = {32: 2e-5, 64: 1e-12, 65: 1e-12}
PLAIN_TOL = {32: 2e-5, 64: 1e-12, 65: 1e-12}
CANCEL_MIN = {32: 8 * 2.0 ** -24 / 2e-5, 64: 1e-3, 65: 8 * 2.0 ** -48 / 1e-12}


def term_scale(U, mesh, order, prm, corr="dg"):
    """RMS over points of B_v, per variable."""
    ops = Ops1D(order, corr)
    Dt = ops.D - np.outer(ops.dhl, ops.lm) - np.outer(ops.dhr, ops.lp)
    G = fr.to_grid(np.asarray(U, dtype=np.float64), mesh, ops.m)
    d = mesh.d
    B = np.abs(acmhd.source(G, prm.T))
    for a in range(d):
        F = np.abs(acmhd.flux(G, a, prm.zeta, prm.nu, prm.T))
        B = B + (2.0 / mesh.h[a]) * fr._apply_along(np.abs(Dt), F, 1 + d + a)
    B = fr.from_grid(B, mesh, ops.m)
    return np.sqrt(np.mean(B * B, axis=(1, 2)))


def errors(R_gpu, R_ref, scale):
    """(scaled error, plain relative error, |R| / scale) per variable.  A
    variable whose terms are all exactly zero (scale 0) must come out exactly
    zero: its scaled error is then 0 or inf."""
    diff = np.sqrt(np.mean((R_gpu - R_ref) ** 2, axis=(1, 2)))
    ref = np.sqrt(np.mean(R_ref ** 2, axis=(1, 2)))
    zero = scale == 0.0
    safe = np.where(zero, 1.0, scale)
    scaled = np.where(zero, np.where(diff == 0.0, 0.0, np.inf), diff / safe)
    return scaled, diff / np.maximum(ref, 1e-300), ref / safe


def assert_parity(R_gpu, R_ref, scale, precision, plain=False, label=""):
    """Scaled bound on every variable; with `plain`, the plain relative bound
    on the variables whose result does not cancel (|R|/|B| >= CANCEL_MIN)."""
    scaled, rel, cancel = errors(R_gpu, R_ref, scale)
    tol = TOL[precision]
    log = os.environ.get("ACMHD_PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"label": label, "precision": precision,
                                "scaled": [float(x) for x in scaled],
                                "plain": [float(x) for x in rel],
                                "cancel": [float(x) for x in cancel]}) + "\n")
    assert np.all(np.isfinite(R_gpu)), f"{label}: non-finite output"
    assert np.all(scaled <= tol), f"{label}: scaled error {scaled.max():.3e} > {tol} ({scaled})"
    if plain:
        sel = cancel >= CANCEL_MIN[precision]   # variables whose result does not cancel
        assert np.all(rel[sel] <= PLAIN_TOL[precision]), (
            f"{label}: plain relative error {rel[sel].max():.3e} > {PLAIN_TOL[precision]} "
            f"(rows {np.nonzero(sel)[0]}, rel {rel}, |R|/|B| {cancel})")
    return scaled, rel


def make_case(n, order, zeta=2.5, nu=1.0 / 1600.0, t_r=5e-3, noise=True, seed=W.NOISE_SEED,
              domain=(-np.pi, np.pi)):
    d = len(n)
    lo, hi = (domain[0],) * d, (domain[1],) * d
    U = W.taylor_green(n, lo, hi, order)
    if noise:
        U = W.add_noise(U, seed=seed)
    return U, fr.Mesh(n, lo, hi), fr.Params(zeta, nu, t_r), lo, hi
