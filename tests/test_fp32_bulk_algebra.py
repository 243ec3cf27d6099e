"""The FP32-bulk mode computes in shifted primitives (p' = p - p_ref,
H' = H - H_ref, T' = T - T_ref about a reference state at rest) from two
FP64 differences, delta rho = rho - rho_ref and delta E = rho e - E_ref.
These are the identities it relies on, checked symbolically:

* p' = (gamma - 1)(delta E - |m|^2 / (2 rho));
* H' = (delta E + p' - H_ref delta rho) / rho;
* T' = (p' / R - T_ref delta rho) / rho;
* the KEP energy flux splits exactly: {rho}{u_n}{H} = {rho}{u_n}{H'} + H_ref
  times the KEP mass flux, so the H_ref part is H_ref times the mass
  equation's right-hand side;
* the p_ref part of the KEP momentum flux is p_ref times the averaged metric,
  whose split-form sum is the discrete metric identity (zero)."""
import pytest

sp = pytest.importorskip("sympy")


def _state(tag):
    rho, E = sp.symbols(f"rho_{tag} E_{tag}", positive=True)
    m = sp.symbols(f"mx_{tag} my_{tag} mz_{tag}", real=True)
    return rho, m, E


def test_shifted_primitives():
    g, R = sp.symbols("gamma R", positive=True)
    rho, m, E = _state("a")
    rho_r, p_r = sp.symbols("rho_r p_r", positive=True)
    E_r = p_r / (g - 1)                       # the reference is at rest
    H_r = (E_r + p_r) / rho_r
    T_r = p_r / (rho_r * R)
    m2 = sum(c * c for c in m)
    p = (g - 1) * (E - m2 / (2 * rho))
    H = (E + p) / rho
    T = p / (rho * R)
    dE, drho = E - E_r, rho - rho_r
    p_s = (g - 1) * (dE - m2 / (2 * rho))
    assert sp.simplify(p_s - (p - p_r)) == 0
    assert sp.simplify((dE + p_s - H_r * drho) / rho - (H - H_r)) == 0
    assert sp.simplify((p_s / R - T_r * drho) / rho - (T - T_r)) == 0


def test_kep_flux_splits_about_the_reference():
    H_r, p_r = sp.symbols("H_r p_r", real=True)
    rL, rR, HL, HR, pL, pR = sp.symbols("rho_L rho_R H_L H_R p_L p_R", real=True)
    uL = sp.symbols("uL0 uL1 uL2", real=True)
    uR = sp.symbols("uR0 uR1 uR2", real=True)
    a = sp.symbols("a0 a1 a2", real=True)      # the averaged metric {Ja}
    avg = lambda x, y: (x + y) / 2
    un = sum(avg(uL[c], uR[c]) * a[c] for c in range(3))
    f_rho = avg(rL, rR) * un
    f_E = avg(rL, rR) * un * avg(HL, HR)
    f_E_shift = avg(rL, rR) * un * avg(HL - H_r, HR - H_r)
    assert sp.expand(f_E - (f_E_shift + H_r * f_rho)) == 0
    for c in range(3):
        f_m = avg(rL, rR) * un * avg(uL[c], uR[c]) + avg(pL, pR) * a[c]
        f_m_shift = avg(rL, rR) * un * avg(uL[c], uR[c]) + avg(pL - p_r, pR - p_r) * a[c]
        assert sp.expand(f_m - (f_m_shift + p_r * a[c])) == 0
