"""The oracle's pins against planted mistakes.

Each case copies the oracle into a scratch directory, plants one plausible
mistake in its C source (a wrong sign, index, factor or dropped term), and
runs tests/test_oracle_pins.py against that copy in a subprocess: at least
one pin must fail.  The unchanged copy must pass, so a failure is the pins'
doing and not the harness's.  Test infrastructure on the CPU only: nothing
here touches the CUDA library.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, exact source text, replacement)
MUTANTS = [
    ("pull_from_x_plus_c",
     "int sx = i - C[q][0], sy = j - C[q][1], sz = k - C[q][2], sq = q;",
     "int sx = i + C[q][0], sy = j + C[q][1], sz = k + C[q][2], sq = q;"),
    ("outlet_copies_known_populations",
     "                    if (C[q][0] < 0)\n                        h->p[(long)q * n + IDX(h, nx - 1, j, k)]",
     "                    if (C[q][0] > 0)\n                        h->p[(long)q * n + IDX(h, nx - 1, j, k)]"),
    ("z_clamped_not_periodic",
     "sz = (sz + nz) % nz;",
     "sz = sz < 0 ? 0 : (sz >= nz ? nz - 1 : sz);"),
    ("slip_wall_mirrors_cz",
     "if (C[r][0] == C[q][0] && C[r][1] == -C[q][1] && C[r][2] == C[q][2]) sq = r;",
     "if (C[r][0] == C[q][0] && C[r][1] == -C[q][1] && C[r][2] == -C[q][2]) sq = r;"),
    ("zou_he_single_outgoing_sum",
     "real rho = (s0 + 2.0 * sm) / (1.0 - uin[0]);",
     "real rho = (s0 + sm) / (1.0 - uin[0]);"),
    ("zou_he_plus_u",
     "real rho = (s0 + 2.0 * sm) / (1.0 - uin[0]);",
     "real rho = (s0 + 2.0 * sm) / (1.0 + uin[0]);"),
    ("fneq_without_half",
     "out[i] = fe[i] + W[i] / (2.0 * CS2 * CS2) * qp;",
     "out[i] = fe[i] + W[i] / (CS2 * CS2) * qp;"),
    ("unknown_fneq_zero",
     "fneq[i] = p[inv] - fe[inv];",
     "fneq[i] = 0.0 * p[inv];"),
    ("smagorinsky_without_sqrt2",
     "18.0 * sqrt(2.0) * c_smag",
     "18.0 * c_smag"),
    ("guo_without_half",
     "(1.0 - 0.5 * s[k]) * mF[k]",
     "(1.0 - s[k]) * mF[k]"),
    ("omega2_d_humieres",
     "    1.0, 1.19, 1.6, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 0.0,",
     "    1.0, 1.19, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 0.0,"),
    ("first_cell_at_one",
     "solve_utau(rabs(uhat), 0.5, h->nu",
     "solve_utau(rabs(uhat), 1.0, h->nu"),
    ("uhat_from_second_cell",
     "real uhat = uw[0] * ex[0] + uw[1] * ex[1] + uw[2] * ex[2];",
     "real uhat = u2[0] * ex[0] + u2[1] * ex[1] + u2[2] * ex[2];"),
    ("tau_w_without_rho",
     "real tw = rw * ut * ut;",
     "real tw = ut * ut;"),
    ("normal_part_kept",
     "tv[a] = u2[a] - un * nrm[a];",
     "tv[a] = u2[a];"),
    ("force_sign_ignored",
     "double sg = RE(uhat) < 0 ? -1.0 : 1.0;",
     "double sg = 1.0;"),
    ("stats_uw_for_uv",
     "s[6] += u * v;",
     "s[6] += u * w;"),
    ("r12_sign_flipped",
     "out[3] = (j + 0.5 < 0.5 * ny) ? -s : s;",
     "out[3] = (j + 0.5 < 0.5 * ny) ? s : -s;"),
    ("j_r_not_centred",
     "real r = (muv - mu * mv) / ur2 - h->Rp[6 * j + 3];",
     "real r = muv / ur2 - h->Rp[6 * j + 3];"),
    ("spectrum_without_dk",
     "* fe * fc * dk;",
     "* fe * fc;"),
    ("no_kolmogorov_factor",
     "real fe = exp(-(12.0 * k / keta) * (12.0 * k / keta));",
     "real fe = 1.0 + 0.0 * k;"),
    ("length_scale_without_wall_limit",
     "h->ell[j] = le * delta * tanh(2.0 * d / (le * delta));",
     "h->ell[j] = le * delta;"),
    ("stg_time_scale_with_k_squared",
     "real xp = (x - h->c.u_bulk * (double)t) * 2.0 * PI_D / (kn * h->maxl);",
     "real xp = (x - h->c.u_bulk * (double)t) * 2.0 * PI_D / (kn * kn * h->maxl);"),
    ("stg_convection_without_u_bulk",
     "real xp = (x - h->c.u_bulk * (double)t) * 2.0 * PI_D / (kn * h->maxl);",
     "real xp = (x - (double)t) * 2.0 * PI_D / (kn * h->maxl);"),
    ("stg_direction_components_swapped",
     "real arg = kn * (d[0] * xp + d[1] * y + d[2] * z) + h->phin[n];",
     "real arg = kn * (d[1] * xp + d[0] * y + d[2] * z) + h->phin[n];"),
    ("sponge_linear_ramp",
     "t0c = tau0 + 3.0 * h->c.sponge_nu * ramp * ramp;",
     "t0c = tau0 + 3.0 * h->c.sponge_nu * ramp;"),
    ("sponge_without_factor_3",
     "t0c = tau0 + 3.0 * h->c.sponge_nu * ramp * ramp;",
     "t0c = tau0 + h->c.sponge_nu * ramp * ramp;"),
]

CONFTEST = '''def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU")
    config.addinivalue_line("markers", "slow: long-running oracle check")
'''


def _run(tmp_path, old, new):
    work = tmp_path / "mut"
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.o", "*.tmp", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "golden")
    shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), work / "test_oracle_pins.py")
    (work / "conftest.py").write_text(CONFTEST)
    src_path = work / "oracle" / "lbm_oracle.c"
    src = src_path.read_text()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src_path.write_text(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(work), ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "test_oracle_pins.py"], cwd=work, env=env, capture_output=True, text=True,
                       timeout=600)
    return r


def test_unchanged_copy_passes(tmp_path):
    r = _run(tmp_path, None, None)
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    r = _run(tmp_path, old, new)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-2000:], r.stderr[-2000:])
