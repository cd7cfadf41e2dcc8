"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the oracle's C
source (a sign, an index, a dropped term, a transposed operand, a wrong constant), rebuilds that copy and
runs the pin suite against it, which must fail.  CPU only; the real oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name: (text of oracle/wn_oracle.c, the mistake that replaces it wherever it occurs)
MUTATIONS = {
    "phase_sign": ("cexp(-2.0 * OR_PI * I * phase)", "cexp(2.0 * OR_PI * I * phase)"),
    "i_power": ("case 1: return -I;", "case 1: return I;"),
    "dropped_w_term": ("w * or_n_minus_1(l[j], m[j]);\n                double complex xi = 1.0;",
                       "0.0;\n                double complex xi = 1.0;"),
    "gaussian_axes_swapped": ("double kx = cos(pa) * v + sin(pa) * u;\n    double ky = -sin(pa) * v + cos(pa) * u;\n    double e",
                              "double kx = cos(pa) * u + sin(pa) * v;\n    double ky = -sin(pa) * u + cos(pa) * v;\n    double e"),
    "hermite_coefficient": ("sqrt((double)n / (n + 1)) * phi[n - 1]", "sqrt((double)(n+1) / (n + 2)) * phi[n - 1]"),
    "frame_transposed": ("s += rj[3 * a + k] * r0[3 * b + k];", "s += rj[3 * k + a] * r0[3 * k + b];"),
    "ra_offset_sign": ("or_uvw_rotation(-dra, dec_j, rj);", "or_uvw_rotation(dra, dec_j, rj);"),
    "peel_conjugate_swapped": ("(g1[0] + I * g1[1]) * conj(g2[0] + I * g2[1])",
                               "conj(g1[0] + I * g1[1]) * (g2[0] + I * g2[1])"),
    "shapelet_scale": ("double K = OR_PI / sqrt(2.0 * log(2.0));\n    double kx = K",
                       "double K = OR_PI / sqrt(log(2.0));\n    double kx = K"),
    "gradient_l_sign": ("(u - w * l[j] / n)", "(u + w * l[j] / n)"),
    "n_minus_1": ("return -r2 / (1.0 + sqrt(1.0 - r2));", "return -r2 / (2.0);"),
    "frame_derivative_dropped": ("g_comp[4 * j + 2] += -2.0 * creal(base * (dxi_x * b1 * dkx_l + dxi_y * b2 * dky_l));",
                                 ";"),
    "frame_derivative_ra_sign": ("double gl = -rh[3 * a + k] * ddra_dl", "double gl = rh[3 * a + k] * ddra_dl"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "wn_oracle.c")).read()
    good, bad = MUTATIONS[name]
    assert src.count(good) >= 1, f"{name}: the text to replace is not in the oracle (update the mutation)"
    ignore = shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__")
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=ignore)
    (tmp_path / "oracle" / "wn_oracle.c").write_text(src.replace(good, bad))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"{name}: every pin passed with the mistake planted\n{r.stdout[-800:]}"
    assert "failed" in r.stdout, r.stdout[-800:] + r.stderr[-800:]
