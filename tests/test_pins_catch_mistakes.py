"""The oracle's pins must catch a plausible mistake anywhere in it.

Each case below plants one mistake (a dropped term, a wrong sign, index or
weight, a transposed operator) in a copy of ``oracle/dg_oracle.c``, builds
the copy in a temporary folder and runs the oracle's pin files
(``tests/test_oracle_*.py``) against it; the mutant passes if every pin still
passes, which fails this test.  The real oracle is never modified.  The pins
stop at the first failure, and the mutants run in parallel, so the whole
check takes well under a minute on a few cores."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dg_oracle.c")

# fast pin files first, so that a caught mutant stops early
PIN_FILES = ["test_oracle_ops.py", "test_oracle_flux.py", "test_oracle_mesh.py", "test_oracle_mms.py",
             "test_oracle_bc.py", "test_oracle_gauss.py", "test_oracle_dg.py"]

# pins that take seconds each (convergence studies)
SLOW = "density_wave_convergence or sod_tube"

# (name, text in the oracle, replacement, which occurrence)
MUTANTS = [
    # operators (Sec. 2.2: LGL nodes, D, Dhat, the split-form operator)
    ("Dhat weight ratio inverted", "o->Dhat[i * n + a] = (real)(-(w[a] / w[i]) * o->Dl[a * n + i]);",
     "o->Dhat[i * n + a] = (real)(-(w[i] / w[a]) * o->Dl[a * n + i]);", 0),
    ("split operator corner sign", "if (i == N && a == N) ds -= 1 / w[N];", "if (i == N && a == N) ds += 1 / w[N];", 0),
    # metrics (curl form)
    ("curl-form sign", "Ja[(v * 3 + i) * 3 + nc] = -curl;", "Ja[(v * 3 + i) * 3 + nc] = curl;", 0),
    ("curl-form index pairing", "mreal curl = mline(n, Dm, V + i2, 3, v, i1) - mline(n, Dm, V + i1, 3, v, i2);",
     "mreal curl = mline(n, Dm, V + i1, 3, v, i1) - mline(n, Dm, V + i2, 3, v, i2);", 0),
    ("Gauss-node metrics left at the LGL nodes", "interp3(n, Ig, Ja, tmp, 9);", "", 0),
    # connectivity
    ("both sides of a face masters", "M->master[ia] = ia < ib;", "M->master[ia] = 1;", 0),
    # point physics
    ("pressure without the 1/2", "q[4] = (P->gamma - 1) * (U[4] - (real)0.5 * (U[1] * q[1]",
     "q[4] = (P->gamma - 1) * (U[4] - (U[1] * q[1]", 0),
    ("temperature without R", "q[5] = q[4] / (U[0] * P->R);", "q[5] = q[4] / U[0];", 0),
    ("KEP flux pressure term dropped", "f[1 + c] = rho * un * u[c] + p * m[c];", "f[1 + c] = rho * un * u[c];", 0),
    ("KEP enthalpy one-sided", "real H = ((UL[4] + qL[4]) / qL[0] + (UR[4] + qR[4]) / qR[0]) / 2;",
     "real H = (UL[4] + qL[4]) / qL[0];", 0),
    ("Roe dissipation sign", "f[v] = (fL[v] + fR[v]) / 2 - D[v] / 2;", "f[v] = (fL[v] + fR[v]) / 2 + D[v] / 2;", 0),
    ("Roe shear waves dropped", "l2 * rt * dut[k];", "0 * dut[k];", 0),
    ("LF with the smaller wave speed", "real lm = lL > lR ? lL : lR;", "real lm = lL < lR ? lL : lR;", 0),
    ("shear stress sign", "real txy = mu * (uy + vx)", "real txy = mu * (uy - vx)", 0),
    ("heat flux sign", "txx * u + txy * v + txz * w + lam * Tx}", "txx * u + txy * v + txz * w - lam * Tx}", 0),
    ("bulk viscosity coefficient", "real txx = mu * (2 * ux - (real)2 / 3 * div);", "real txx = mu * (2 * ux - div);", 0),
    ("Sutherland exponent", "return P->mu * (real)1.4042 * th * RSQRT(th) / (th + (real)0.4042);",
     "return P->mu * (real)1.4042 * th / (th + (real)0.4042);", 0),
    # the LGL operator (Eq. dgsem, Eq. lifting)
    ("lifting operator transposed", "o->Dhat[i * n + a] * Jaa[x] * w->q[", "o->Dhat[a * n + i] * Jaa[x] * w->q[", 0),
    ("lifting slave sign", "w->g[(e2 * n3 + vS) * 12 + qv * 3 + x] -= fl", "w->g[(e2 * n3 + vS) * 12 + qv * 3 + x] += fl", 0),
    ("lifting times J", "for (int k = 0; k < 12; ++k) w->g[(e * n3 + v) * 12 + k] /= M->J[e * n3 + v];",
     "for (int k = 0; k < 12; ++k) w->g[(e * n3 + v) * 12 + k] *= M->J[e * n3 + v];", 0),
    ("split metrics not averaged", "real m[3] = {(Jai[0] + Jaa[0]) / 2, (Jai[1] + Jaa[1]) / 2, (Jai[2] + Jaa[2]) / 2};",
     "real m[3] = {Jaa[0], Jaa[1], Jaa[2]};", 0),
    ("split operator transposed", "+= o->Dsplit[i * n + a] * fs[k];", "+= o->Dsplit[a * n + i] * fs[k];", 0),
    ("viscous volume sign", "w->B[(e * n3 + v) * 5 + k] -= o->Dhat[i * n + a] * fv[k];",
     "w->B[(e * n3 + v) * 5 + k] += o->Dhat[i * n + a] * fv[k];", 0),
    ("viscous surface flux one-sided", "fs[k] -= (fvM[k] + fvS[k]) / 2;", "fs[k] -= fvM[k];", 0),
    ("surface slave sign", "w->B[(e2 * n3 + vS) * 5 + k] -= fs[k]", "w->B[(e2 * n3 + vS) * 5 + k] += fs[k]", 0),
    ("surface weight", "w->B[(e * n3 + vM) * 5 + k] += fs[k] / o->w[(f % 2) ? n - 1 : 0];",
     "w->B[(e * n3 + vM) * 5 + k] += fs[k] / o->w[1];", 1),
    ("ApplyJac sign", "Ut[x] = -(w->Bc[x] + w->B[x]) / M->J[e * n3 + v];",
     "Ut[x] = (w->Bc[x] + w->B[x]) / M->J[e * n3 + v];", 0),
    # shock capturing (Sec. 2.3)
    ("indicator on density alone", "s[v] = qe[v * 6 + 0] * qe[v * 6 + 4];", "s[v] = qe[v * 6 + 0];", 0),
    ("indicator threshold degree", "RPOW((real)(N + 1), (real)0.25)", "RPOW((real)(N), (real)0.25)", 0),
    ("indicator second-highest mode dropped", "real e2 = totN1 > 0 ? mj[N - 1] / totN1 : 0;", "real e2 = 0;", 0),
    ("FV interface metrics without weights", "Jh[i + 1][c] = Jh[i][c] + o->w[i] * dj;", "Jh[i + 1][c] = Jh[i][c] + dj;", 0),
    ("FV right-node weight", "vfv[vr * 5 + k] -= fb[k] * s / o->w[i + 1];", "vfv[vr * 5 + k] -= fb[k] * s / o->w[i];", 0),
    ("blend without 1 - alpha", "= (1 - al) * w->Bc[(e * n3 + v) * 5 + k] + al * vfv[v * 5 + k];",
     "= w->Bc[(e * n3 + v) * 5 + k] + al * vfv[v * 5 + k];", 0),
    # boundary conditions and sponge
    ("wall pressure sign", "for (int c = 0; c < 3; ++c) fs[1 + c] = p * nu[c] * s;",
     "for (int c = 0; c < 3; ++c) fs[1 + c] = -p * nu[c] * s;", 0),
    ("adiabatic wall keeps the heat flux", "if (type == BC_WALL_ADIABATIC) gw[9] = gw[10] = gw[11] = 0;", "", 0),
    ("isothermal wall lifts the inner T", "qs[0] = b[1]; qs[1] = b[2]; qs[2] = b[3]; qs[3] = b[4];",
     "qs[0] = b[1]; qs[1] = b[2]; qs[2] = b[3]; qs[3] = q[5];", 0),
    ("outflow energy without the 1/2", "Ue[4] = b[1] / (P->gamma - 1) + (real)0.5 * (U[1] * q[1]",
     "Ue[4] = b[1] / (P->gamma - 1) + (U[1] * q[1]", 0),
    ("sponge sign", "if (M->sponge_sigma) Ut[x] -= M->sponge_sigma", "if (M->sponge_sigma) Ut[x] += M->sponge_sigma", 0),
    # manufactured-solution source (Sec. 5.1)
    ("MMS advection sign", "Q[0] = (3 - P->src_a) * c;", "Q[0] = (3 + P->src_a) * c;", 0),
    ("MMS heat conduction order", "Q[4] += 3 * lam * g1 / P->R * w * w * sn;", "Q[4] += 3 * lam * g1 / P->R * w * sn;", 0),
    # Gauss-Legendre nodes
    ("GL face value from the wrong end", "const real* L = (f % 2) ? M->o.Lp : M->o.Lm;",
     "const real* L = (f % 2) ? M->o.Lm : M->o.Lp;", 0),
    ("GL SurfInt without 1/w", "+= sgn_add * val[c] * L[a] / M->o.w[a];", "+= sgn_add * val[c] * L[a];", 0),
    ("GL volume operator transposed", "w->Bc[(e * n3 + v) * 5 + k] += o->Dhat[i * n + a] * fc[k];",
     "w->Bc[(e * n3 + v) * 5 + k] += o->Dhat[a * n + i] * fc[k];", 0),
    # time integration and time step (Sec. 2.2)
    ("stage time dropped", "f(ctx, U, t + rk->C[s] * dt, Ut);", "f(ctx, U, t, Ut);", 0),
    # the fourteen-stage table: one digit mistyped in A, B and c
    ("fourteen-stage A digit", "-2.0837094552574054", "-2.0837094562574054", 0),
    ("fourteen-stage B digit", "0.1524043173028741", "0.1524043173029741", 0),
    ("fourteen-stage c digit", "0.8190890835352128", "0.8190890835352728", 0),
    ("stage update without the register", "U[x] = U[x] + rk->B[s] * dU[x];", "U[x] = U[x] + rk->B[s] * dt * Ut[x];", 0),
    ("CFL step without (N+1)^2", "real dt = P->cfl * 2 / (np1 * np1 * lc);", "real dt = P->cfl * 2 / (np1 * lc);", 0),
    ("CFL sound speed times |Ja|^2", "+ c * RSQRT(nj2);", "+ c * nj2;", 0),
    ("viscous step factor fixed at 4/3", "real kv = (real)4 / 3 > P->gamma / P->Pr ? (real)4 / 3 : P->gamma / P->Pr;",
     "real kv = (real)4 / 3;", 0),
    ("viscous step with (N+1)^2", "real dv = P->dfl * 4 / (np1 * np1 * np1 * np1 * lv);",
     "real dv = P->dfl * 4 / (np1 * np1 * lv);", 0),
    ("second stage register index", "dU[x] = (s == 0 ? 0 : rk->A[s] * dU[x]) + dt * Ut[x];",
     "dU[x] = (s == 0 ? 0 : rk->A[s - 1] * dU[x]) + dt * Ut[x];", 0),
    # nodes, weights and the Lagrange basis
    ("Legendre recurrence coefficient", "oreal p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;",
     "oreal p2 = ((2 * k + 1) * x * p1 - (k - 1) * p0) / k;", 0),
    ("LGL weights with N^2", "w[j] = 2 / ((oreal)N * (N + 1) * P * P);", "w[j] = 2 / ((oreal)N * N * P * P);", 0),
    ("GL weights without 1 - x^2", "w[j] = 2 / ((1 - t * t) * dP * dP);", "w[j] = 2 / (dP * dP);", 0),
    ("derivative matrix transposed", "D[i * n + j] = s;", "D[j * n + i] = s;", 0),
    ("modal basis not normalised", "V[i * n + m] = sqrtl((oreal)(2 * m + 1) / 2) * P;", "V[i * n + m] = P;", 0),
    # connectivity and the Gauss-node face terms
    ("partner face node transposed", "M->nbr_node[ef * n2 + p + n * q] = found;",
     "M->nbr_node[ef * n2 + q + n * p] = found;", 0),
    ("GL face normal sign", "real sgn = (f % 2) ? 1 : -1;", "real sgn = (f % 2) ? -1 : 1;", 2),
    ("GL face value weights", "for (int c = 0; c < ncomp; ++c) out[c] += L[a] * fld[(e * n3 + va) * ncomp + c];",
     "for (int c = 0; c < ncomp; ++c) out[c] += fld[(e * n3 + va) * ncomp + c] / M->n;", 0),
    ("GL metric Jacobian at the LGL nodes", "interp3(n, Ig, dx, tmp, 9);", "", 0),
    ("GL lifting slave sign", "surf_spread(M, w->g, 12, e2, f2, a2 % n, a2 / n, fl, -1);",
     "surf_spread(M, w->g, 12, e2, f2, a2 % n, a2 / n, fl, 1);", 0),
    ("GL surface slave sign", "surf_spread(M, w->B, 5, e2, f2, a2 % n, a2 / n, fs, -1);",
     "surf_spread(M, w->B, 5, e2, f2, a2 % n, a2 / n, fs, 1);", 0),
    # boundary states
    ("prescribed state ignored", "for (int k = 0; k < 5; ++k) Ue[k] = b[1 + k];", "for (int k = 0; k < 5; ++k) Ue[k] = U[k];", 0),
    ("slip wall lifts the full velocity", "for (int c = 0; c < 3; ++c) qs[c] = q[1 + c] - un * nu[c];",
     "for (int c = 0; c < 3; ++c) qs[c] = q[1 + c];", 0),
    # physics details
    ("Sutherland constant", "(th + (real)0.4042)", "(th + (real)1.4042)", 0),
    ("MMS momentum source without pressure", "Q[k] = (3 - P->src_a) * c + g1 * (2 * rho - (real)1.5) * c;",
     "Q[k] = (3 - P->src_a) * c;", 0),
    # diagnostics
    ("kinetic energy without 1/2", "ek += wq * r * v2 / 2;", "ek += wq * r * v2;", 0),
    ("kinetic energy rate mass-term sign", "- v2 * ut[0] / 2", "+ v2 * ut[0] / 2", 0),
    ("vorticity component sign", "real wx = d[7] - d[5]", "real wx = d[7] + d[5]", 0),
    ("vorticity from the wrong gradient", "wz = d[3] - d[1];", "wz = d[3] - d[2];", 0),
    ("dilatational rate without 4/3", "out[1] = (double)(4 * P.mu * ed / (3 * vol));",
     "out[1] = (double)(P.mu * ed / vol);", 0),
    ("dissipation without the viscosity weight", "real r = viscosity(&P, q[5]) / P.mu;", "real r = 1;", 0),
]


def _mutant_source(old, new, occ):
    with open(SRC) as f:
        s = f.read()
    at = -1
    for _ in range(occ + 1):
        at = s.find(old, at + 1)
        assert at >= 0, f"planted text not found: {old!r} (occurrence {occ})"
    return s[:at] + new + s[at + len(old):]


def _run(case, tmp):
    name, old, new, occ = case
    d = os.path.join(tmp, str(MUTANTS.index(case)))
    os.makedirs(d)
    src = os.path.join(d, "dg_oracle.c")
    with open(src, "w") as f:
        f.write(_mutant_source(old, new, occ))
    env = dict(os.environ, DG_ORACLE_SOURCE=src, DG_ORACLE_BUILD=os.path.join(d, "build"),
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
           *[os.path.join(ROOT, "tests", p) for p in PIN_FILES]]
    try:
        # the quick pins first; the slow convergence studies only if those pass
        for sel in ("not (" + SLOW + ")", SLOW):
            p = subprocess.run(cmd + ["-k", sel], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
            if p.returncode != 0:
                break
    except subprocess.TimeoutExpired:
        return name, "timeout", ""
    tail = (p.stdout + p.stderr).strip().splitlines()
    first = next((ln for ln in tail if ln.startswith("FAILED ")), tail[-1] if tail else "")
    return name, p.returncode, first


def test_planted_text_is_unique_where_it_must_be():
    for name, old, new, occ in MUTANTS:
        assert old != new, name
        _mutant_source(old, new, occ)


def test_every_planted_mistake_fails_a_pin():
    pytest.importorskip("numpy")
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    workers = max(1, min(len(MUTANTS), cores, 16))   # each worker is a pytest process of ~150 MB
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(workers) as ex:
            results = list(ex.map(lambda c: _run(c, tmp), MUTANTS))
    survived = [(n, how) for n, rc, how in results if rc == 0]
    broken = [(n, rc, how) for n, rc, how in results if rc not in (0, 1) and not (isinstance(rc, int) and rc < 0)]
    assert not broken, broken          # a mutant that did not build, or a pytest usage error
    assert not survived, survived
