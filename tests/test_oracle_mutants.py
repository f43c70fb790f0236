"""Planted mistakes in copies of the oracle source must each fail a pin.

Every mutant is a plausible slip (a dropped term, a wrong sign or index, a
transposed operand, a wrong tie rule) written into a temporary copy of
``oracle/fsr_oracle.c`` on the CPU; the committed oracle is never touched.
"""
import pytest

import oracle
import oracle_pins as P

MUTANTS = {
    "shift_row_sign": ("int i = (k - u >= 0) ? k - u : S + k - u;",
                       "int i = (k + u < S) ? k + u : k + u - S;"),
    "shift_col_sign": ("int j = (l - v >= 0) ? l - v : S + l - v;",
                       "int j = (l + v < S) ? l + v : l + v - S;"),
    "update_no_gamma": ("const double are = P->gamma * pre, aim = P->gamma * pim;",
                        "const double are = pre, aim = pim;"),
    "model_no_S2": ("Gre[idx] += P->gamma * pre * (double)SS;\n        Gim[idx] += P->gamma * pim * (double)SS;",
                    "Gre[idx] += P->gamma * pre;\n        Gim[idx] += P->gamma * pim;"),
    "p_over_S2": ("const double pre = Rre[idx] / W0, pim = Rim[idx] / W0;",
                  "const double pre = Rre[idx] / (double)SS, pim = Rim[idx] / (double)SS;"),
    "update_conj": ("Rim[k * S + l] -= are * d + aim * c;",
                    "Rim[k * S + l] -= are * d - aim * c;"),
    "update_real_sign": ("Rre[k * S + l] -= are * c - aim * d;",
                         "Rre[k * S + l] -= are * c + aim * d;"),
    "dft_transposed": ("            Xre[k * S + l] = sr;\n            Xim[k * S + l] = si;",
                       "            Xre[l * S + k] = sr;\n            Xim[l * S + k] = si;"),
    "dft_sign": ("Tim[t] = -sin(a);", "Tim[t] = sin(a);"),
    "no_freq_weight": ("double obj = wf[i] * (Rre[i] * Rre[i] + Rim[i] * Rim[i]);",
                       "double obj = (Rre[i] * Rre[i] + Rim[i] * Rim[i]);"),
    "tie_highest": ("if (obj > best) {", "if (obj >= best) {"),
    "centre_S_over_2": ("double c = (double)(S - 1) / 2.0;", "double c = (double)S / 2.0;"),
    "wf_no_sqrt2": ("double b = 1.0 - sqrt(2.0) * r;", "double b = 1.0 - r;"),
    "wf_kt_unfolded": ("double kt = half - fabs((double)k - half);",
                       "double kt = fabs((double)k - half);"),
    "known_not_copied": ("else val = kn[m * S + n] ? f[m * S + n] : gre[m * S + n];",
                         "else val = gre[m * S + n];"),
    "tiling_transposed": ("const long by = b / nbx, bx = b % nbx;",
                          "const long bx = b / nby, by = b % nby;"),
    "tiling_origin": ("const long y0 = by * B - L, x0 = bx * B - L;",
                      "const long y0 = by * B - L + 1, x0 = bx * B - L;"),
    "inverse_sign": ("double c = Tre[t], d = -Tim[t];", "double c = Tre[t], d = Tim[t];"),
    "inverse_scale": ("if (o->gre) o->gre[m * S + n] = sr / (double)SS;",
                      "if (o->gre) o->gre[m * S + n] = sr;"),
    "unknown_read": ("x[i] = scale[i] > 0.0 ? f[i] * w[i] : 0.0;", "x[i] = f[i] * w[i];"),
    "weight_everywhere": ("w[i] = scale[i] > 0.0 ? scale[i] * w0[i] : 0.0;", "w[i] = w0[i];"),
    "scale_ignored": ("w[i] = scale[i] > 0.0 ? scale[i] * w0[i] : 0.0;", "w[i] = scale[i] > 0.0 ? w0[i] : 0.0;"),
    # the conjugate-pair ablation
    "pair_model_not_conjugate": ("Gim[sel_conj] -= cim * (double)SS;", "Gim[sel_conj] += cim * (double)SS;"),
    "pair_second_shift_sign": ("const int d2 = ((k + su) % S) * S + (l + sv) % S;",
                               "const int d2 = ((k + S - su) % S) * S + (l + sv) % S;"),
    "pair_update_diff_sign": ("ur = cre * sr - cim * di;", "ur = cre * sr + cim * di;"),
    "pair_selfconj_doubled": ("if (sel_conj == sel) {", "if (0) {"),
    # the re-use form (reconstructed pixels of earlier blocks)
    "reuse_no_delta": ("                        sc = delta;", "                        sc = 1.0;"),
    "reuse_own_block": ("} else if ((y / B) * nbx + (x / B) < b) {", "} else if ((y / B) * nbx + (x / B) <= b) {"),
    "reuse_column_order": ("} else if ((y / B) * nbx + (x / B) < b) {",
                           "} else if ((x / B) * nby + (y / B) < bx * nby + by) {"),
    "reuse_origin": ("        const long x0 = bx * B - L;", "        const long x0 = bx * B - L + 1;"),
    "reuse_value_from_input": ("                        v = src[y * Wd + x];",
                               "                        v = (double)img[y * pitch + x];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = oracle.build_variant(src.replace(old, new), str(tmp_path), "mut_" + name)
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(lib)
        except Exception as e:  # an assertion, or a numpy error on garbage
            failed.append((pin.__name__, type(e).__name__))
    assert failed, f"mutant {name} passed every pin"
