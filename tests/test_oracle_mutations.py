"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong sign, a swapped table
entry, a transposed operand) in a copy of the oracle's C source, builds it,
and runs the pin suite against that build in a child process: the suite must
fail.  The mistakes are planted on the CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

MUTATIONS = {
    "equilibrium_drops_quadratic": ("(cu * cu) / (2.0 * cs2 * cs2)", "0.0"),
    "equilibrium_linear_sign": ("1.0 + cu / cs2", "1.0 - cu / cs2"),
    "lattice_c7_c8_swapped": ("static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};",
                              "static const int CX[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};"),
    "weights_axis_diag_swapped": ("1.0 / 9.0, 1.0 / 9.0,\n                             1.0 / 36.0, 1.0 / 36.0",
                                  "1.0 / 36.0, 1.0 / 36.0,\n                             1.0 / 9.0, 1.0 / 9.0"),
    "bgk_rate_inverted": ("g[i] = g[i] - (g[i] - feq[i]) / s->tau;", "g[i] = g[i] - (g[i] - feq[i]) * (1.0 - 1.0 / s->tau);"),
    "stream_pushes_instead_of_pulls": ("int sx = x - CX[i], sy = y - CY[i];", "int sx = x + CX[i], sy = y + CY[i];"),
    "moments_ux_from_jy": ("m[1] = jx / rho;", "m[1] = jy / rho;"),
    "mirror_sign": ("g[i] = feq[i] + (g[o] - feq[o]);", "g[i] = feq[i] - (g[o] - feq[o]);"),
    "mirror_uses_own_eq": ("g[i] = feq[i] + (g[o] - feq[o]);", "g[i] = feq[o] + (g[o] - feq[i]);"),
    "gradient_sign": ("mp[c] = mb[c] - s->gamma * dn;", "mp[c] = mb[c] + s->gamma * dn;"),
    "gradient_drops_corner_length": ("dn = (mb[c] - m1[c]) / len;", "dn = (mb[c] - m1[c]);"),
    "blend_transposed": ("mc[c] = (1.0 - s->beta) * mp[c] + s->beta * s->m0[c];",
                         "mc[c] = s->beta * mp[c] + (1.0 - s->beta) * s->m0[c];"),
    "doubly_unknown_zeroed": ("      g[i] = feq[i];\n  }", "      g[i] = 0.0;\n  }"),
    "correction_without_weights": ("g[i] -= WT[i] * (drho + s->kappa", "g[i] -= (1.0 / 9.0) * (drho + s->kappa"),
    "correction_ignores_kappa": ("(drho + s->kappa * (CX[i] * djx", "(drho + 1.0 * (CX[i] * djx"),
    "second_order_stencil_sign": ("(3.0 * mb[c] - 4.0 * m1[c] + m2[c])", "(3.0 * mb[c] - 4.0 * m1[c] - m2[c])"),
    "mrt_gram_schmidt_skips_projection": ("v[i] -= num / den * s->M[b][i];", "v[i] -= 0.0 * num / den * s->M[b][i];"),
    "mrt_inverse_not_normalised": ("s->Minv[i][a] = s->M[a][i] / n2;", "s->Minv[i][a] = s->M[a][i];"),
    "mrt_inverse_transposed": ("d += s->Minv[i][a] * r[a];", "d += s->Minv[a][i] * r[a];"),
    "mrt_relaxes_away_from_equilibrium": ("r[a] = s->mrt_s[a] * (m[a] - meq[a]);",
                                          "r[a] = s->mrt_s[a] * (meq[a] - m[a]);"),
    "corner_mean_takes_one_edge_twice": ("mc[c] = 0.5 * (mx[c] + my[c]);", "mc[c] = 0.5 * (mx[c] + mx[c]);"),
    "corner_mode_ignored": ("if (s->corner_mode == 1 && nxn != 0 && nyn != 0) {", "if (0) {"),
    "corner_edge_normal_keeps_diagonal": ("predict_blend(s, x, y, nxn, 0, mx);", "predict_blend(s, x, y, nxn, nyn, mx);"),
    "velocity_edge_ignored": ("      mc[1] = s->uw[side][0];", "      mc[1] = mc[1];"),
    "velocity_edge_axes_swapped": ("      mc[2] = s->uw[side][1];", "      mc[2] = s->uw[side][0];"),
}


# mistakes in the storage emulation (a test instrument of the oracle), caught
# by its own pins in test_oracle_storage.py
STORAGE_MUTATIONS = {
    "bf16_truncates": ("b += 0x7fffu + ((b >> 16) & 1u);", "b += 0u;"),
    "f16_unscaled": ("(double)(_Float16)(float)(v * 4096.0) / 4096.0", "(double)(_Float16)(float)(v)"),
    "rounds_absolute_populations": ("F(s, buf, i, x, y) = r[i] + q_store(F(s, buf, i, x, y) - r[i], s->store_fmt);",
                                    "F(s, buf, i, x, y) = q_store(F(s, buf, i, x, y), s->store_fmt);"),
    "far_field_shift_ignored": ("  if (s->store_ff)\n    or_equilibrium", "  if (0)\n    or_equilibrium"),
}


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, source, tmp_path):
    _planted_mistake_fails(MUTATIONS, name, source, tmp_path, "test_oracle_pins.py")


@pytest.mark.parametrize("name", sorted(STORAGE_MUTATIONS))
def test_planted_storage_mistake_fails_a_pin(name, source, tmp_path):
    _planted_mistake_fails(STORAGE_MUTATIONS, name, source, tmp_path, "test_oracle_storage.py")


def _planted_mistake_fails(table, name, source, tmp_path, pins):
    old, new = table[name]
    assert source.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "lbm_oracle_mut.c"
    mutated.write_text(source.replace(old, new))
    so = tmp_path / "liblbm_oracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=gnu99", "-fPIC", "-shared", "-o", str(so),
                           str(mutated), "-lm"])
    env = dict(os.environ, LBM_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught mutation {name}:\n{r.stdout[-2000:]}"
