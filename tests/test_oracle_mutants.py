"""Sensitivity of the oracle pins: each plausible mistake planted in a copy of the oracle source
(a dropped term, a wrong sign, a swapped index or operand, the paper's own flagged typo) must make
at least one pin of oracle_pins.py fail. CPU only; the mutants are built in a temporary folder."""
import pytest

import oracle
from oracle_pins import PINS

MUTANTS = [
    # Sec. 2.3: the flagged typo u^- x t in the last HC line
    ("hc_typo", "cross3(up, tv, up_x_t);", "cross3(um, tv, up_x_t);"),
    ("hc_sigma_sign", "double sigma = gm * gm - tau2;", "double sigma = gm * gm + tau2;"),
    ("hc_half_kick", "for (int c = 0; c < 3; c++) unew[c] = up[c] + h * E[c] + up_x_t[c];",
     "for (int c = 0; c < 3; c++) unew[c] = up[c] + up_x_t[c];"),
    ("push_charge_sign", "double h = -Q_E * dt / (2.0 * M_ELEC);", "double h = Q_E * dt / (2.0 * M_ELEC);"),
    ("push_full_drift", "xi[c] = xh[c] + 0.5 * dt * v[3 * i + c];", "xi[c] = xh[c] + dt * v[3 * i + c];"),
    # eq:LW_E / eq:LW_B
    ("lw_drop_accel", "E[c] = pref * (c2mv2 * vp[c] + acc[c]);", "E[c] = pref * (c2mv2 * vp[c]);"),
    ("lw_accel_order", "cross3(eta, vp_x_a, acc);", "cross3(vp_x_a, eta, acc);"),
    ("lw_inner_cross", "cross3(vp, a, vp_x_a);", "cross3(a, vp, vp_x_a);"),
    ("lw_b_transposed", "cross3(nhat, E, nxE);", "cross3(E, nhat, nxE);"),
    ("lw_c2_plus_v2", "double c2mv2 = C_LIGHT * C_LIGHT - dot3(v, v);", "double c2mv2 = C_LIGHT * C_LIGHT + dot3(v, v);"),
    ("lw_vprime_sign", "C_LIGHT * nhat[2] - v[2]};", "C_LIGHT * nhat[2] + v[2]};"),
    ("lw_power", "(4.0 * PI * EPS0 * eta_vp * eta_vp * eta_vp)", "(4.0 * PI * EPS0 * eta_vp * eta_vp * R)"),
    # eq:dt
    ("dt_c1_sign", "double C1 = 2.0 * (dot3(d, v1) - C_LIGHT * C_LIGHT * T1);",
     "double C1 = 2.0 * (-dot3(d, v1) - C_LIGHT * C_LIGHT * T1);"),
    ("dt_other_root", "*dt_out = ra < rb ? ra : rb;", "*dt_out = ra < rb ? rb : ra;"),
    ("dt_c0_sign", "double C0 = C_LIGHT * C_LIGHT * T1 * T1 - dot3(d, d);",
     "double C0 = dot3(d, d) - C_LIGHT * C_LIGHT * T1 * T1;"),
    # eq:linear
    ("linear_v_weights", "v[c] = v1[c] * (1.0 - df) + v2[c] * df;", "v[c] = v1[c] * df + v2[c] * (1.0 - df);"),
    ("linear_a_sign", "a[c] = (v2[c] - v1[c]) / (t2 - t1);", "a[c] = (v1[c] - v2[c]) / (t2 - t1);"),
    ("linear_w_from_w2", "for (int c = 0; c < 3; c++) w[c] = w1[c] + v1[c] * dt;",
     "for (int c = 0; c < 3; c++) w[c] = hist_w(h, k1 + (k1 < n), j)[c] + v1[c] * dt;"),
    # Sec. 2.2 bracket
    ("bisect_flipped", "if (node_test(r, t, h->T[m], hist_w(h, m, j)))", "if (!node_test(r, t, h->T[m], hist_w(h, m, j)))"),
    ("shortcut_wrong_node", "if (!node_test(r, t, h->T[n - 1], hist_w(h, n - 1, j))) {",
     "if (!node_test(r, t, h->T[n - 1], hist_w(h, n, j))) {"),
    ("half_width_test", "double ct = C_LIGHT * (t - tk);", "double ct = 0.5 * C_LIGHT * (t - tk);"),
    ("special_keeps_accel", "      a[c] = 0.0;\n", "      a[c] = v1[c] * 1e3;\n"),
    # eq:mid and the half-step field point (comparison variants)
    ("mid_w_from_w1", "w[c] = (w1[c] + w2[c]) / 2.0;", "w[c] = w1[c];"),
    ("mid_v_from_v1", "v[c] = (v1[c] + v2[c]) / 2.0;", "v[c] = v1[c];"),
    ("mid_a_sign", "a[c] = (v2[c] - v1[c]) / span;", "a[c] = (v1[c] - v2[c]) / span;"),
    ("mid_tr_at_t1", "*tr = (t1 + t2) / 2.0;", "*tr = t1;"),
    ("half_full_time", "T[n + 1] = T[n] + 0.5 * dt;", "T[n + 1] = T[n] + dt;"),
    ("half_no_drift", "Wp[3 * i + c] = Wn[3 * i + c] + 0.5 * dt * (u[3 * i + c] / g0);", "Wp[3 * i + c] = Wn[3 * i + c];"),
    ("half_present_point", "st = orc_self_fields_ex(N, T, W, V, n + 1, D,", "st = orc_self_fields_ex(N, T, W, V, n, D,"),
    # Sec. 2.4 adaptive time step
    ("adapt_target_velocity_old_slot", "const double* vi = hist_v(&h, n, i);", "const double* vi = hist_v(&h, k0, i);"),
    ("adapt_cutoff_ignored", "if (R < eta_allow) continue;", "if (R < 0.0) continue;"),
    ("adapt_vrel_sum", "double dv[3] = {vi[0] - v[0], vi[1] - v[1], vi[2] - v[2]};",
     "double dv[3] = {vi[0] + v[0], vi[1] + v[1], vi[2] + v[2]};"),
    ("adapt_no_clamp_low", "return fmin(dt_max, fmax(dt_min, dt));", "return fmin(dt_max, dt);"),
    ("adapt_present_separation", "double eta[3] = {r[0] - w[0], r[1] - w[1], r[2] - w[2]};\n      double R",
     "double eta[3] = {r[0] - hist_w(&h, n, j)[0], r[1] - hist_w(&h, n, j)[1], r[2] - hist_w(&h, n, j)[2]};\n      double R"),
    # Sec. 2.7 stage switch
    ("energy_includes_rest_mass", "double Ei = uu / (gamma_of_u(u + 3 * i) + 1.0) * M_ELEC * C_LIGHT * C_LIGHT;",
     "double Ei = (uu / (gamma_of_u(u + 3 * i) + 1.0) + 1.0) * M_ELEC * C_LIGHT * C_LIGHT;"),
    ("energy_weight_squared", "csum_add(&num, wi * Ei);", "csum_add(&num, wi * wi * Ei);"),
    ("switch_not_armed", "run = (armed && fabs(r) < eps) ? run + 1 : 0;", "run = (fabs(r) < eps) ? run + 1 : 0;"),
    ("switch_signed_rate", "run = (armed && fabs(r) < eps) ? run + 1 : 0;", "run = (armed && r < eps) ? run + 1 : 0;"),
    ("switch_time_base", "double r = (E[n] - E[n - 1]) / (T[n] - T[n - 1]);", "double r = (E[n] - E[n - 1]) / (T[n] - T[0]);"),
    ("switch_first_of_hold", "if (found < 0 && run >= hold) found = n;", "if (found < 0 && run >= hold) found = n - hold + 1;"),
    # Sec. 2.6 dipole
    ("dipole_factor", "B[c] = k * (3.0 * Mr * rhat[c] - M[c]);", "B[c] = k * (2.0 * Mr * rhat[c] - M[c]);"),
    ("dipole_power", "double k = MU0 / (4.0 * PI) / (r * r * r);", "double k = MU0 / (4.0 * PI) / (r * r);"),
]


@pytest.mark.parametrize("name,orig,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, orig, repl, tmp_path):
    src = open(oracle._SRC).read()
    assert src.count(orig) == 1, f"snippet for mutant {name} not found exactly once"
    mpath = tmp_path / f"{name}.c"
    mpath.write_text(src.replace(orig, repl))
    lib = oracle.load(oracle.compile_lib(str(mpath), str(tmp_path / f"lib{name}.so"), openmp=False))
    for pin in PINS:
        try:
            pin(lib)
        except (AssertionError, oracle.OracleError, FloatingPointError, ValueError, ZeroDivisionError):
            return
    pytest.fail(f"mutant {name} passed every pin")
