"""Each pin must catch a plausible mistake: plant one in a copy of the oracle
source (a dropped term, a wrong sign, index or operand), build that copy, run
the CPU pin suite against it and require a failure.  Mistakes are planted in
the oracle only, on the CPU."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_hllc.py", "test_oracle_riemann.py", "test_oracle_scheme.py",
         "test_oracle_weno.py", "test_oracle_rad.py", "test_oracle_advect.py")]

# (name, original text, planted text)
MUTANTS = [
    ("minmod picks the larger slope", "return (a <= b) ? a : b;", "return (a <= b) ? b : a;"),
    ("left face state sign", "qL[f] = W[1][f] + 0.5 * dqi;", "qL[f] = W[1][f] - 0.5 * dqi;"),
    ("right face state sign", "qR[f] = W[2][f] - 0.5 * dqi1;", "qR[f] = W[2][f] + 0.5 * dqi1;"),
    ("right face uses left slope", "qR[f] = W[2][f] - 0.5 * dqi1;", "qR[f] = W[2][f] - 0.5 * dqi;"),
    ("pressure kinetic sign", "W[4] = (gamma - 1.0) * (U[4] - kin);",
     "W[4] = (gamma - 1.0) * (U[4] + kin);"),
    ("kinetic energy drops w", "double kin = 0.5 * rho * (u * u + v * v + w * w);",
     "double kin = 0.5 * rho * (u * u + v * v);"),
    ("sound speed without gamma", "double cL = sqrt(gamma * pL / rL);",
     "double cL = sqrt(pL / rL);"),
    ("contact speed pressure sign", "(pR - pL + rL", "(pL - pR + rL"),
    ("contact speed denominator", "/ (rL * (SL - uL) - rR * (SR - uR));",
     "/ (rL * (SL - uL) + rR * (SR - uR));"),
    ("star energy sign", "(Sstar + p / (r * (SK - u)))", "(Sstar - p / (r * (SK - u)))"),
    ("star energy term dropped",
     "Us[4] = fac * (UK[4] / r + (Sstar - u) * (Sstar + p / (r * (SK - u))));",
     "Us[4] = fac * (UK[4] / r);"),
    ("momentum flux without p", "F[1] = rho * un * un + p;", "F[1] = rho * un * un;"),
    ("energy flux without p", "F[4] = (E + p) * un;", "F[4] = E * un;"),
    ("face energy drops t2",
     "double E = p / (gamma - 1.0) + 0.5 * rho * (un * un + t1 * t1 + t2 * t2);",
     "double E = p / (gamma - 1.0) + 0.5 * rho * (un * un + t1 * t1);"),
    ("reflect index", "return m < 0 ? -1 - m : 2 * n - 1 - m;",
     "return m < 0 ? -m : 2 * n - 1 - m;"),
    ("reflect keeps momentum", "if (flip) out[1 + d] = -out[1 + d];",
     "if (flip) out[1 + d] = out[1 + d];"),
    ("periodic wrap off by one", "return r < 0 ? r + n : r;", "return r < 0 ? r + n - 1 : r;"),
    ("outflow copies the wrong cell", "if (bc == BC_OUTFLOW) return m < 0 ? 0 : n - 1;",
     "if (bc == BC_OUTFLOW) return m < 0 ? 1 : n - 1;"),
    ("stage 2 half dt", "Uout[q] = 0.5 * U0[q] + 0.5 * (Ucur[q] + dt * L[q]);",
     "Uout[q] = 0.5 * U0[q] + 0.5 * (Ucur[q] + 0.5 * dt * L[q]);"),
    ("stage 2 weights", "Uout[q] = 0.5 * U0[q] + 0.5 * (Ucur[q] + dt * L[q]);",
     "Uout[q] = 0.25 * U0[q] + 0.75 * (Ucur[q] + dt * L[q]);"),
    ("divergence uses dx for every axis",
     "(Ff[f * nfaces + fhi] - Ff[f * nfaces + flo]) / g->dx[d];",
     "(Ff[f * nfaces + fhi] - Ff[f * nfaces + flo]) / g->dx[0];"),
    ("y sweep uses the x normal", "{{1, 2, 3}, {2, 1, 3}, {3, 1, 2}}",
     "{{1, 2, 3}, {1, 2, 3}, {3, 1, 2}}"),
    ("z sweep uses the y normal", "{{1, 2, 3}, {2, 1, 3}, {3, 1, 2}}",
     "{{1, 2, 3}, {2, 1, 3}, {2, 1, 3}}"),
    ("rate without sound speed", "r += (fabs(W[1 + d]) + cs) / g.dx[d];",
     "r += (fabs(W[1 + d])) / g.dx[d];"),
    ("rate uses dx for every axis", "r += (fabs(W[1 + d]) + cs) / g.dx[d];",
     "r += (fabs(W[1 + d]) + cs) / g.dx[0];"),
    ("face flux shifted by one cell", "c[d] -= 1;                        /* left cell of the face */",
     ""),
    ("HLLC side swapped", "double SK = (Sstar >= 0.0) ? SL : SR;",
     "double SK = (Sstar >= 0.0) ? SR : SL;"),
    ("Davis bound mixes sides", "double SL = fmin(uL - cL, uR - cR);",
     "double SL = fmin(uL - cL, uL - cR);"),
    ("stencil shifted", "fetch_cons(g, U, d, i, j, k, s - 1, Uc);",
     "fetch_cons(g, U, d, i, j, k, s - 2, Uc);"),
    ("exact shock density", "W3[0] = rL * (ps / pL + gm) / (gm * ps / pL + 1.0);",
     "W3[0] = rL * (ps / pL + gm) / (gm * ps / pL - 1.0);"),
    ("exact fan velocity", "W3[1] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + xi);",
     "W3[1] = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL - xi);"),
    ("exact shock pressure function", "*f = (p - pK) * q;", "*f = (p + pK) * q;"),
    ("Heun weights", "Unew[q] = Un[q] + dt * (0.5 * k1[q] + 0.5 * k2[q]);",
     "Unew[q] = Un[q] + dt * (0.5 * k1[q] + 0.5 * k1[q]);"),
    # second scheme: WENO5-Z face states and the HLL flux
    ("WENO linear weight d1", "double a1 = 0.6 * (1.0 + tau / (b1 + WENO_EPS));",
     "double a1 = 0.5 * (1.0 + tau / (b1 + WENO_EPS));"),
    ("WENO middle candidate stencil", "double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;",
     "double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[4]) / 6.0;"),
    ("WENO right candidate sign", "double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;",
     "double p2 = (2.0 * v[2] + 5.0 * v[3] + v[4]) / 6.0;"),
    ("WENO tau from the wrong indicators", "double tau = fabs(b0 - b2);",
     "double tau = fabs(b0 - b1);"),
    ("WENO indicator slope term", "t0 = v[0] - 4.0 * v[1] + 3.0 * v[2];",
     "t0 = v[0] - 4.0 * v[1] + 2.0 * v[2];"),
    ("WENO indicator curvature weight", "double b2 = 13.0 / 12.0 * s2 * s2 + 0.25 * t2 * t2;",
     "double b2 = s2 * s2 + 0.25 * t2 * t2;"),
    ("WENO weights not normalised", "return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);",
     "return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1);"),
    ("WENO right state not mirrored",
     "double r[5] = {W[5][f], W[4][f], W[3][f], W[2][f], W[1][f]};",
     "double r[5] = {W[1][f], W[2][f], W[3][f], W[4][f], W[5][f]};"),
    ("WENO stencil shifted", "fetch_cons(g, U, d, i, j, k, s - 2, Uc);",
     "fetch_cons(g, U, d, i, j, k, s - 3, Uc);"),
    ("HLL dissipation sign",
     "F[f] = (SR * FL[f] - SL * FR[f] + SL * SR * (UR[f] - UL[f])) / (SR - SL);",
     "F[f] = (SR * FL[f] - SL * FR[f] - SL * SR * (UR[f] - UL[f])) / (SR - SL);"),
    ("HLL Davis bound", "double SL = fmin(WL[1] - cL, WR[1] - cR);",
     "double SL = fmin(WL[1] - cL, WR[1] + cR);"),
    # radiative heating / cooling exchange
    ("exchange source sign", "double f = x - e - dt * k * (Etot - x - aT4);",
     "double f = x - e + dt * k * (Etot - x - aT4);"),
    ("exchange T^4 as T^3", "double aT4 = arad * (T * T) * (T * T);",
     "double aT4 = arad * (T * T) * T;"),
    ("exchange rate without density", "double k = c * kappa * rho;", "double k = c * kappa;"),
    ("radiation energy update sign", "Er[q] = Er[q] + (e - x);", "Er[q] = Er[q] - (e - x);"),
    ("exchange ignores kinetic energy", "U[4 * N + q] = x + kin;", "U[4 * N + q] = x;"),
    # radiation energy advection
    ("Rusanov dissipation sign", "return 0.5 * (EL * uL + ER * uR) - 0.5 * a * (ER - EL);",
     "return 0.5 * (EL * uL + ER * uR) + 0.5 * a * (ER - EL);"),
    ("Rusanov speed from one side", "double a = fmax(fabs(uL), fabs(uR));", "double a = fabs(uL);"),
    ("advection velocity from the wrong axis", "u[s] = W[1 + d];", "u[s] = W[1];"),
    ("advected E states not mirrored",
     "er[5] = {e[5], e[4], e[3], e[2], e[1]};", "er[5] = {e[1], e[2], e[3], e[4], e[5]};"),
]


def _run_mutant(args):
    idx, (name, old, new), tmp = args
    src = open(os.path.join(ROOT, "oracle", "hard_oracle.c")).read()
    assert old in src, f"mutation site of '{name}' not found"
    cpath = os.path.join(tmp, f"m{idx}.c")
    with open(cpath, "w") as fh:
        fh.write(src.replace(old, new, 1))
    so = oracle.compile_oracle(cpath, os.path.join(tmp, f"m{idx}.so"))
    env = dict(os.environ, HARD_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       env=env, capture_output=True, text=True, cwd=ROOT)
    return name, r.returncode


# mistakes planted in the flux-limited diffusion oracle (oracle/fld.py)
FLD_MUTANTS = [
    ("limiter denominator", "(2.0 + R) / (6.0 + 3.0 * R + R * R)",
     "(2.0 + R) / (6.0 + 2.0 * R + R * R)"),
    ("face coefficient from one side", "w = 0.5 * (D + Dn) * dt / (dxyz[d] * dxyz[d])",
     "w = 0.5 * (D + D) * dt / (dxyz[d] * dxyz[d])"),
    ("face weight not over dx^2", "w = 0.5 * (D + Dn) * dt / (dxyz[d] * dxyz[d])",
     "w = 0.5 * (D + Dn) * dt / dxyz[d]"),
    ("gradient without the factor 2", "/ (2.0 * dxyz[d])", "/ dxyz[d]"),
    ("coefficient without rho", "return c * flux_limiter(R) / (kappa * rho)",
     "return c * flux_limiter(R) / kappa"),
    ("R without kappa", "R = np.sqrt(grad2) / (rho * kappa * E)", "R = np.sqrt(grad2) / (rho * E)"),
    ("off-diagonal sign", "vals += [-w.ravel(), -w.ravel()]", "vals += [w.ravel(), w.ravel()]"),
]


def _run_fld_mutant(args):
    idx, (name, old, new), tmp = args
    src = open(os.path.join(ROOT, "oracle", "fld.py")).read()
    assert old in src, f"mutation site of '{name}' not found"
    path = os.path.join(tmp, f"fld_m{idx}.py")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new, 1))
    env = dict(os.environ, HARD_FLD_PATH=path)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_fld.py"),
                        "-x", "-q", "-p", "no:cacheprovider"],
                       env=env, capture_output=True, text=True, cwd=ROOT)
    return name, r.returncode


def test_every_planted_fld_mistake_is_caught(tmp_path):
    if os.environ.get("HARD_FLD_PATH"):
        pytest.skip("already running against a planted copy")
    jobs = [(i, m, str(tmp_path)) for i, m in enumerate(FLD_MUTANTS)]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run_fld_mutant, jobs))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins did not catch: {survivors}"


def test_every_planted_mistake_is_caught(tmp_path):
    if os.environ.get("HARD_ORACLE_LIB"):
        pytest.skip("already running against a planted copy")
    jobs = [(i, m, str(tmp_path)) for i, m in enumerate(MUTANTS)]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run_mutant, jobs))
    survivors = [name for name, rc in results if rc == 0]
    assert not survivors, f"pins did not catch: {survivors}"
