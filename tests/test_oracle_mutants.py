"""Each pin must catch a plausible mistake planted in a copy of the oracle.

Every case below edits one expression of ``oracle/lf_oracle.c`` in a
temporary copy, compiles it, and runs the pins named beside it: at least one
must fail.  This shows that the pins fix the oracle's arithmetic, not only
that the oracle agrees with itself.  CPU only.
"""
import pytest

import oracle
import pins

MUTANTS = [
    ("x_tol uses p instead of 1/p",
     "p->xtol_c + p->xtol_p / pmom", "p->xtol_c + p->xtol_p * pmom", ["pin_window_edges"]),
    ("asymmetry on the wrong side",
     "float a_left = ((qpos && mu) || (!qpos && !mu))", "float a_left = ((!qpos && mu) || (qpos && !mu))",
     ["pin_window_edges"]),
    ("stereo correction with the wrong sign",
     "centre = (xn + tx_f * (g->z[l] - g->z[n])) - yl * g->dxdy[l];",
     "centre = (xn + tx_f * (g->z[l] - g->z[n])) + yl * g->dxdy[l];", ["pin_window_edges"]),
    ("window lower edge exclusive", "while (i < hi && x[i] < v) ++i;", "while (i < hi && x[i] <= v) ++i;",
     ["pin_window_edges_inclusive"]),
    ("window upper edge exclusive", "while (i < hi && !(x[i] > v)) ++i;", "while (i < hi && x[i] < v) ++i;",
     ["pin_window_edges_inclusive"]),
    ("x-layer extension cut four times T_x", "if (dx * dx < p->T_x) cd->hit[l] = h;",
     "if (dx * dx < 4.0f * p->T_x) cd->hit[l] = h;", ["pin_extension_T_x"]),
    ("x-layer extension cut inclusive", "if (dx * dx < p->T_x) cd->hit[l] = h;",
     "if (dx * dx <= 1.005f * p->T_x) cd->hit[l] = h;", ["pin_extension_T_x"]),
    ("stereo extension cut four times T_uv", "if (dx * dx < T_uv) cd->hit[l] = h;",
     "if (dx * dx < 4.0f * T_uv) cd->hit[l] = h;", ["pin_extension_T_uv"]),
    ("stereo extension cut without the slope term", "T_uv = fmaxf(p->T_uv_min, T_uv);\n    for",
     "T_uv = p->T_uv_min;\n    for", ["pin_extension_T_uv"]),
    ("window cap not symmetric", "start = c - cap / 2;", "start = c - cap / 4;", ["pin_window_cap"]),
    ("window cap not clamped at the low end", "if (start < lo) start = lo;", "", ["pin_window_cap"]),
    ("closest-hit tie to the higher index", "if (best < 0 || d < bd)", "if (best < 0 || d <= bd)",
     ["pin_closest_tie"]),
    ("K multiplies the whole extrapolation",
     "float x1_exp = z1 * tx_d + (x0 - tx_d * z0) * K;",
     "float x1_exp = (z1 * tx_d + (x0 - tx_d * z0)) * K;", ["pin_triplet_chi2_K"]),
    ("T_triplet inclusive and doubled", "if (!(chi2 < p->T_triplet)) continue;",
     "if (!(chi2 <= 2.0f * p->T_triplet)) continue;", ["pin_triplet_chi2_K"]),
    ("keeps the largest chi2",
     "if (p->chi2 < q->chi2) return -1;\n    if (p->chi2 > q->chi2) return 1;",
     "if (p->chi2 < q->chi2) return 1;\n    if (p->chi2 > q->chi2) return -1;", ["pin_top_n"]),
    ("bending filter inverted",
     "int ok = (bend > 0.0f) ? (d > 0.0f) : (d < 0.0f);",
     "int ok = (bend > 0.0f) ? (d < 0.0f) : (d > 0.0f);", ["pin_bending_filter", "pin_closed_form"]),
    ("magnet tolerance without the slope term",
     "float tol = tol_base + p->magtol_tx * fabsf(tx_d);", "float tol = tol_base;",
     ["pin_magnet_tolerance"]),
    ("extension searches the triplet layers",
     "static const int CFG_MISSING[2][3] = {{3, 7, 11}, {0, 4, 8}};",
     "static const int CFG_MISSING[2][3] = {{0, 4, 8}, {3, 7, 11}};", ["pin_closed_form"]),
    ("C(n) table reversed", "* p->C_n[n - 9];", "* p->C_n[12 - n];", ["pin_known_residual_Q"]),
    ("nDoF_x = n - 2", "(qx / (float)(n - 3)", "(qx / (float)(n - 2)", ["pin_known_residual_Q"]),
    ("Q_y dropped", "qy = qy + (ry * ry) / p->T_y;", "qy = qy + 0.0f * ry;", ["pin_known_residual_Q"]),
    ("stereo residual against the input y", "float r = hx[h] - (xf - yf * hdxdy[h]);",
     "float r = hx[h] - (xf - (s->ys + s->tys * (hz[h] - g->z_state)) * hdxdy[h]);",
     ["pin_known_residual_Q"]),
    ("T_Q doubled", "if (!(Q < p->T_Q))", "if (!(Q < 2.0f * p->T_Q))", ["pin_T_Q"]),
    ("t_y cut against the sum", "fabsf(ty_fit - s->tys) < p->T_ty", "fabsf(ty_fit + s->tys) < p->T_ty",
     ["pin_ty_cut", "pin_closed_form"]),
    ("y from the hit minus the model", "float y = (model_x(A, T, C, u, D) - hx[h]) / hdxdy[h];",
     "float y = (hx[h] - model_x(A, T, C, u, D)) / hdxdy[h];", ["pin_closed_form", "pin_ty_cut"]),
    ("binary64 model without dRatio", "double f[3] = {1.0, dz, dz * dz * (1.0 + dR * dz)};",
     "double f[3] = {1.0, dz, dz * dz};", ["pin_closed_form"]),
    ("q/p ignores the polarity", "cd->state[5] = (tx - s->txs) / ((float)g->polarity * g->kappa);",
     "cd->state[5] = (tx - s->txs) / g->kappa;", ["pin_closed_form_md"]),
    ("polynomial q/p without the slope normalisation", "float sf = tx_f / sqrtf((1.0f + tx_f * tx_f) + ty_f * ty_f);",
     "float sf = tx_f;", ["pin_qop_polynomial"]),
    ("polynomial q/p with dSlope reversed", "float ds = tx_f - tx_i;", "float ds = tx_i - tx_f;",
     ["pin_qop_polynomial"]),
    ("polynomial q/p coefficients with t_x and t_y swapped",
     "acc = acc + p->qop_c[i][j] * (txp[k] * typ[m]);", "acc = acc + p->qop_c[i][j] * (txp[m] * typ[k]);",
     ["pin_qop_polynomial"]),
    ("polynomial q/p ignores the polarity", "return (sf - si) / ((float)g->polarity * F);", "return (sf - si) / F;",
     ["pin_qop_polynomial_md"]),
    ("x refit skipped", "A = A + ((c00 * b0 + c01 * b1) + c02 * b2) / dt;", "A = A + 0.0f * dt;",
     ["pin_fit32_vs_fit64"]),
    ("stereo-hit-per-station requirement dropped",
     "if (!st_uv[0] || !st_uv[1] || !st_uv[2]) { cd->status = CS_UV_STATION; return; }", "",
     ["pin_invariants", "pin_known_residual_Q"]),
    ("pack sorts x descending",
     "if (p->x < q->x) return -1;\n    if (p->x > q->x) return 1;",
     "if (p->x < q->x) return 1;\n    if (p->x > q->x) return -1;", ["pin_pack_lexsort"]),
    ("pack keeps negative zero", "ox[o] = x[r] + 0.0f;", "ox[o] = x[r];", ["pin_pack_lexsort"]),
    ("compaction skips the last track of an event",
     "for (int32_t t = trk_offsets[e]; t < trk_offsets[e + 1]; ++t)\n            if (found[t])",
     "for (int32_t t = trk_offsets[e]; t + 1 < trk_offsets[e + 1]; ++t)\n            if (found[t])",
     ["pin_compact"]),
    # no-UT variant
    ("no-UT windows swap sides", "float xmin = side ? centre - p->x_overlap : centre - tol;",
     "float xmin = side ? centre - tol : centre - p->x_overlap;", ["pin_no_ut_window_edges"]),
    ("no-UT overlap on the wrong side of the line", "float xmax = side ? centre + tol : centre + p->x_overlap;",
     "float xmax = side ? centre + tol : centre - p->x_overlap;", ["pin_no_ut_window_edges"]),
    ("no-UT assumed momentum the looser threshold", "return fminf(ip_p, ip_pt);", "return fmaxf(ip_p, ip_pt);",
     ["pin_no_ut_window_edges"]),
    ("no-UT pT threshold with tan(theta)", "float sin_theta = sqrtf(t2) / sqrtf(1.0f + t2);",
     "float sin_theta = sqrtf(t2);", ["pin_no_ut_window_edges"]),
    ("no-UT c3 term linear in ty", "float b = (ty * ty) * (c[3] + tx * (c[4] + c[5] * tx));",
     "float b = ty * (c[3] + tx * (c[4] + c[5] * tx));", ["pin_no_ut_window_edges"]),
    ("no-UT c4 and c5 swapped", "(c[3] + tx * (c[4] + c[5] * tx))", "(c[3] + tx * (c[5] + c[4] * tx))",
     ["pin_no_ut_window_edges"]),
    ("no-UT c6 term without t_x", "float d = ip * (c[6] * tx + c[7] * ip);",
     "float d = ip * (c[6] + c[7] * ip);", ["pin_no_ut_window_edges"]),
    ("no-UT u/v windows with the x tolerance", "            tol = p->uv_tol;\n", "            tol = x_tol;\n",
     ["pin_no_ut_window_edges"]),
    ("no-UT extrapolation with the kick", "centre = s->xs + s->txs * (g->z[l] - g->z_state);",
     "centre = x_extrap(g, s, l);", ["pin_no_ut_window_edges"]),
    ("no-UT extension in the other side's windows", "&Ws[trips[r].side]", "&Ws[1 - trips[r].side]",
     ["pin_no_ut_closed_form", "pin_no_ut_closed_form_md"]),
    ("no-UT side ranked after the configuration",
     "if (p->side != q->side) return p->side < q->side ? -1 : 1;\n    if (p->cfg != q->cfg) return p->cfg < q->cfg ? -1 : 1;",
     "if (p->cfg != q->cfg) return p->cfg < q->cfg ? -1 : 1;\n    if (p->side != q->side) return p->side < q->side ? -1 : 1;",
     ["pin_no_ut_overlap"]),
    ("no-UT only one side seeded", "for (int side = 0; side < n_sides; ++side) {",
     "for (int side = n_sides - 1; side < n_sides; ++side) {", ["pin_no_ut_closed_form", "pin_no_ut_overlap"]),
]


@pytest.mark.parametrize("name,old,new,pin_names", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, pin_names, tmp_path):
    src = oracle.source()
    assert src.count(old) == 1, "mutation anchor not found once: %r" % old
    orc = oracle.variant(src.replace(old, new), str(tmp_path), "mutant")
    caught = []
    for pn in pin_names:
        try:
            getattr(pins, pn)(orc)
        except AssertionError:
            caught.append(pn)
    assert caught, "no pin caught: %s" % name
