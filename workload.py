"""Seeded synthetic workloads for the Fokker-Planck QTT solver.

This module only draws and packs input parameters (grid bits, coefficients,
random velocity-mode wavevectors/phases, the time step).  It holds none of
the method's arithmetic: both the CUDA library and the CPU oracle receive the
same parameter dictionary and evaluate the velocity field, the initial PDF and
the operators themselves.

Workloads (one PDF f(phi1, phi2; x1, x2, x3) on [0,1]^2 x [0, 2pi)^3):
  small   2^4 points per dimension (20 QTT sites, 2^20 cells), chi_max 32, 50 steps
  medium  2^6 points per dimension (30 sites, 2^30 cells), chi_max 64, 200 steps
  large   2^8 points per dimension (40 sites, 2^40 cells), chi_max 128, 500 steps
Velocity: u1 = tanh(x2 - pi) plus 4 random Fourier modes of amplitude 0.1,
each mode adding a*sin(k.x + theta) to one component c with k_c = 0 (so the
field is divergence-free).  Diffusivity 1e-2, Omega = 1, Da = 1, artificial
composition-space dissipation D_phi = 4e-3 * Omega.
Initial PDF: normalised Gaussian of standard deviation 0.05 centred at
(phi1, phi2) = (1, 0) for x2 > pi and at (0, 1) otherwise, blended by
w(x2) = (1 + tanh((x2 - pi)/0.2))/2.
"""
from __future__ import annotations

import copy
import math

import numpy as np

PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3, "bf16x10": 4}

WORKLOADS = {
    "small": dict(bits=4, chi_max=32, steps=50),
    "medium": dict(bits=6, chi_max=64, steps=200),
    "large": dict(bits=8, chi_max=128, steps=500),
}


def draw_velocity_modes(seed: int, n_modes: int = 4, amp: float = 0.1, kmax: int = 2):
    """Random Fourier modes: component c, integer wavevector k with k[c] = 0 and
    the other two entries in [-kmax, kmax], not both zero; phase ~ U[0, 2pi)."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(n_modes):
        c = int(rng.integers(0, 3))
        while True:
            k = [int(v) for v in rng.integers(-kmax, kmax + 1, size=3)]
            k[c] = 0
            if any(k):
                break
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        modes.append(dict(comp=c, k=k, phase=theta, amp=float(amp)))
    return modes


def cfl_dt(bits, omega, da, gamma, d_phi, u_bound, cfl=0.2):
    """Time step from the stability limits of the explicit scheme, using the
    bound u_bound >= max_x sum_i |u_i| (advection), Omega + Da (composition
    drift speed on [0,1]^2) and the two diffusion numbers."""
    hx = min(2.0 * math.pi / 2 ** b for b in bits[2:])
    hp = min(1.0 / 2 ** b for b in bits[:2])
    lims = [hp / max(omega + da, 1e-300)]
    if u_bound > 0:
        lims.append(hx / u_bound)
    if gamma > 0:
        lims.append(hx * hx / (6.0 * gamma))
    if d_phi > 0:
        lims.append(hp * hp / (4.0 * d_phi))
    return cfl * min(lims)


def velocity_bound(p: dict) -> float:
    """Upper bound of sum_i |u_i| for the stability rule: the shear (flow 0) or
    the Taylor-Green vortex and jet (flow 1: |u1| <= 2 u0, |u2| <= u0,
    |u3| <= 2 u0), plus the seeded modes."""
    base = 5.0 * abs(p.get("u0", 1.0)) if p.get("flow", 0) == 1 else abs(p["shear_amp"])
    return base + sum(abs(m["amp"]) for m in p["umodes"])


def make_paper_params(bits: int = 5, chi: int = 64, seed: int = 0, precision: str = "fp64", **overrides) -> dict:
    """The paper's own flow case (Materials and Methods, Flow case definition)
    on [0, 2 pi)^3: jet through a Taylor-Green vortex (Eq. velField, u0 = 1),
    the Gaussian step-function initial PDF (Eq. initPDF: centres (3/4, 1/4)
    inside the band 1/4 <= x1/l0 < 3/4 and (1/4, 3/4) outside, width 1/8) with
    tanh edges of width 0.1, gamma = u0 l0 / Pe with Pe = 10^3, Omega = 1,
    Da = 0 (the case with a numerically exact moment equation), D_phi = mu
    Omega with mu = 4e-3.  The subgrid fields gamma_SGS(x) and Omega_mix(x) are
    constants here (gamma_SGS = 0, Omega_mix = Omega)."""
    kw = dict(flow=1, u0=1.0, ic_kind=1, ic_sigma=0.125, ic_c_hi=[0.75, 0.25], ic_c_lo=[0.25, 0.75],
              ic_blend_width=0.1, gamma=2.0 * math.pi / 1.0e3, omega=1.0, da=0.0, d_phi=4e-3, shear_amp=0.0,
              umodes=[])
    kw.update(overrides)
    return make_params({"bits": bits, "chi_max": chi, "steps": 1}, seed=seed, precision=precision, **kw)


def make_params(workload: str = "small", seed: int = 0, precision: str = "fp64",
                **overrides) -> dict:
    """Parameter dictionary for one PDF.  Keys mirror the C struct qtt_params."""
    w = WORKLOADS[workload] if isinstance(workload, str) else dict(workload)
    K = w["bits"]
    p = dict(
        bits=[K] * 5,
        chi_max=w["chi_max"],
        svd_rel_tol=1e-14 if precision in ("fp64", "bf16x10") else 1e-7,
        precision=PRECISIONS[precision],
        omega=1.0,
        da=1.0,
        gamma=1e-2,
        d_phi=4e-3,
        shear_amp=1.0,
        umodes=draw_velocity_modes(seed),
        ic_sigma=0.05,
        ic_blend_width=0.2,
        ic_c_hi=[1.0, 0.0],
        ic_c_lo=[0.0, 1.0],
        icmodes=[],
        rk_variant=0,
        steps=w.get("steps", 1),
        seed=seed,
    )
    p.update(copy.deepcopy(overrides))
    if "dt" not in overrides:
        ub = velocity_bound(p)
        p["dt"] = cfl_dt(p["bits"], p["omega"], p["da"], p["gamma"], p["d_phi"], ub)
    return p


# Batched configuration: independent PDFs of uneven grid and chi.
BATCH = {"n": 256, "bits": (5, 6, 7), "chi": (16, 32, 64, 96), "da_log10": (-1.0, 1.0), "omega": (0.5, 2.0),
         "steps": 100, "mu": 4e-3}


def make_batch_params(n: int = BATCH["n"], seed: int = 0, precision: str = "fp32") -> list:
    """n instance parameter dictionaries: Da log-uniform in [0.1, 10], Omega
    uniform in [0.5, 2], bits per dimension uniform in {5, 6, 7}, chi_max
    uniform in {16, 32, 64, 96}, drawn from numpy default_rng(seed); instance
    i takes the velocity modes of seed i; the artificial dissipation is
    D_phi = mu Omega with mu = 4e-3; dt from the stability rule."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        da = float(10.0 ** rng.uniform(*BATCH["da_log10"]))
        omega = float(rng.uniform(*BATCH["omega"]))
        K = int(rng.choice(BATCH["bits"]))
        chi = int(rng.choice(BATCH["chi"]))
        w = {"bits": K, "chi_max": chi, "steps": BATCH["steps"]}
        out.append(make_params(w, seed=i, precision=precision, da=da, omega=omega, d_phi=BATCH["mu"] * omega))
    return out



def draw_ic_modes(seed: int, n_modes: int = 16, kmax: int = 2):
    """Initial-condition modulation modes f0 *= 1 + sum_m b_m cos(q_m . x + psi_m):
    integer q_m in [-kmax, kmax]^3 without 0, psi_m ~ U[0, 2pi), b_m = 0
    (the nominal point of the gradient)."""
    rng = np.random.default_rng(seed + 7919)
    modes = []
    for _ in range(n_modes):
        while True:
            q = [int(v) for v in rng.integers(-kmax, kmax + 1, size=3)]
            if any(q):
                break
        modes.append(dict(k=q, phase=float(rng.uniform(0.0, 2.0 * math.pi)), amp=0.0))
    return modes


# Adjoint configuration: 2^6 points per dimension, chi 64, FP32 form, the
# gradient in Omega, Da, gamma, 4 velocity and 16 initial-condition amplitudes.
ADJOINT = {"bits": 6, "chi_max": 64, "steps": 200, "ckpt_every": 20, "n_ic": 16}


def make_adjoint_params(seed: int = 0, precision: str = "fp32") -> dict:
    p = make_params({"bits": ADJOINT["bits"], "chi_max": ADJOINT["chi_max"], "steps": ADJOINT["steps"]}, seed=seed,
                    precision=precision)
    p["icmodes"] = draw_ic_modes(seed, ADJOINT["n_ic"])
    return p


def make_truncation_trains(nsites: int, ell: int, chi: int, seed: int = 11):
    """Inputs of the truncation backward at a step's sizes: X as nsites cores
    [r_n][2][r_{n+1}] with r_n = min(2^n, 2^(nsites-n), ell), the first
    nsites-1 random isometries (orthonormal columns of a Gaussian matrix, the
    form the zip-up leaves) and a Gaussian last core; the cotangent as a
    Gaussian train of bonds min(2^n, 2^(nsites-n), chi).  Returns (r, x, s, y)
    with x and y the cores flattened one after another."""
    rng = np.random.default_rng(seed)
    r = [min(2 ** n, 2 ** (nsites - n), ell) for n in range(nsites + 1)]
    s = [min(2 ** n, 2 ** (nsites - n), chi) for n in range(nsites + 1)]
    xc = [np.linalg.qr(rng.standard_normal((2 * r[n], r[n + 1])))[0] for n in range(nsites - 1)]
    xc.append(rng.standard_normal((2 * r[nsites - 1], 1)))
    yc = [rng.standard_normal(s[n] * 2 * s[n + 1]) for n in range(nsites)]
    return r, np.concatenate([c.ravel() for c in xc]), s, np.concatenate(yc)
