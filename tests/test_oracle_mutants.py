"""The oracle's pins catch plausible mistakes.

Each mutant below plants one mistake (a dropped term, a flipped sign, a transposed
operand, a missing correction) in a copy of the oracle on the CPU; the two pin suites
(test_oracle.py and test_oracle_mapping.py, copied beside it with what they import) then
run against that copy in a fresh interpreter.  Every mutant must fail at least one pin,
and the unmutated copy none: a mistake anywhere in the oracle's arithmetic shows up
before the oracle is trusted to judge the CUDA path.
"""
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_SUITES = ("test_oracle.py", "test_oracle_mapping.py", "test_oracle_mask.py")

# name: (file in oracle/, text, its replacement)
MUTANTS = {
    # projection (Sec. II-A pi_m, the covariance of Sec. I)
    "Jacobian x-depth term dropped": ("gs_oracle.c", "g->J[2] = -cam->fx * g->tan_c[0] / z;", "g->J[2] = 0.0;"),
    "conic off-diagonal sign": ("gs_oracle.c", "pr->conic[1] = -S01 / det;", "pr->conic[1] = S01 / det;"),
    "camera covariance transposed": ("gs_oracle.c", "mat3_mul(R, g->Sigma, RS);\n    mat3_transpose(R, Rt);\n"
                                     "    mat3_mul(RS, Rt, g->Sigma_c);",
                                     "mat3_transpose(R, Rt);\n    mat3_mul(Rt, g->Sigma, RS);\n"
                                     "    mat3_mul(RS, R, g->Sigma_c);"),
    # compositing (Eqs. 2-4)
    "transmittance update": ("gs_oracle.c", "const double z = pr->xc[2];\n        const double Tn = T * (1.0 - alpha);",
                             "const double z = pr->xc[2];\n        const double Tn = T * (1.0 - 0.5 * alpha);"),
    "depth weighted by T only": ("gs_oracle.c", "D += z * w;", "D += z * T;"),
    # reverse compositing and chain rule
    "behind-colour update": ("gs_oracle.c", "B[ch] = c->alpha * v[ch] + (1.0 - c->alpha) * B[ch];",
                             "B[ch] = c->alpha * v[ch] + B[ch];"),
    "pose rotation sign (mean part)": ("gs_oracle.c", "pose6[0] += xc[1] * dxc[2] - xc[2] * dxc[1];",
                                       "pose6[0] -= xc[1] * dxc[2] - xc[2] * dxc[1];"),
    "pose rotation sign (covariance part)": ("gs_oracle.c", "pose6[1] += -2.0 * M[2];", "pose6[1] += 2.0 * M[2];"),
    "quaternion normalisation partial": ("gs_oracle.c", "dq[k] = (dqn[k] - g.qn[k] * proj) / g.qnorm;",
                                         "dq[k] = (dqn[k] + g.qn[k] * proj) / g.qnorm;"),
    "log-scale chain factor dropped": ("gs_oracle.c", "dls[j] = ds * g.s[j];", "dls[j] = ds;"),
    # decoupled pose update
    "pose Adam bias correction dropped": ("gs_oracle.c", "const double mh = *m / bc1, vh = *v / bc2;",
                                          "const double mh = *m, vh = *v / bc2;"),
    "pose rotation step direction": ("gs_oracle.c", "dq[1] = -step[0] * s;", "dq[1] = step[0] * s;"),
    # the FP32-facing parts: the depth key and the ambiguity mask
    "depth key from the wrong row": ("gs_oracle.c", "return fmaf(Rf[6], m0, fmaf(Rf[7], m1, fmaf(Rf[8], m2, tf[2])));",
                                     "return fmaf(Rf[3], m0, fmaf(Rf[4], m1, fmaf(Rf[5], m2, tf[2])));"),
    "depth key without translation": ("gs_oracle.c", "return fmaf(Rf[6], m0, fmaf(Rf[7], m1, fmaf(Rf[8], m2, tf[2])));",
                                      "return fmaf(Rf[6], m0, fmaf(Rf[7], m1, Rf[8] * m2));"),
    "alpha margin 100x too wide": ("gs_oracle.c", "return fmax(p->amb_alpha, e->dexp);",
                                   "return fmax(100.0 * p->amb_alpha, e->dexp);"),
    "t_min margin 30x too wide": ("gs_oracle.c", "return fabs(Tn - p->t_min) <= fmax(p->amb_t, eT) * p->t_min;",
                                  "return fabs(Tn - p->t_min) <= 30.0 * fmax(p->amb_t, eT) * p->t_min;"),
    "camera-transform error dropped from the margin": ("gs_oracle.c", "+ sqrt(gx * gx + gy * gy) * pr->dmu;",
                                                       ";"),
    # map side (Sec. III-A, III-C) and metrics (Sec. IV)
    "unprojection rotation transposed": ("mapping.py", "means = (xc - t) @ R  #", "means = (xc - t) @ R.T  #"),
    "map Adam bias correction dropped": ("mapping.py", "m_hat = mk / (1.0 - beta1 ** step)", "m_hat = mk"),
    "removal threshold inverted": ("mapping.py", "reshape(-1) >= thr", "reshape(-1) <= thr"),
    "PSNR amplitude factor": ("metrics.py", "10.0 * np.log10(1.0 / mse)", "20.0 * np.log10(1.0 / mse)"),
    "camera centre without transpose": ("metrics.py", "return -_rotation(p[:4]).T @ p[4:7]",
                                        "return -_rotation(p[:4]) @ p[4:7]"),
    "MS-SSIM window width": ("metrics.py", "g = np.exp(-x * x / (2.0 * sigma * sigma))",
                             "g = np.exp(-x * x / (sigma * sigma))"),
}


def _copy(src_dir, dst_dir, names):
    os.makedirs(dst_dir, exist_ok=True)
    for n in names:
        s = os.path.join(src_dir, n)
        if os.path.isdir(s):
            shutil.copytree(s, os.path.join(dst_dir, n))
        else:
            shutil.copy(s, os.path.join(dst_dir, n))


def run_pins(work, mutant=None):
    """Copy the oracle (planting `mutant`) and the pin suites into `work`, run the suites
    in a fresh interpreter and return (failed, passed, pytest's output)."""
    _copy(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
          ("__init__.py", "gs_oracle.c", "mapping.py", "metrics.py"))
    _copy(os.path.join(ROOT, "tests"), os.path.join(work, "tests"), ("conftest.py", "golden", "mask_model.py") + PIN_SUITES)
    _copy(os.path.join(ROOT, "paper_2408_05635_gb300"), os.path.join(work, "paper_2408_05635_gb300"),
          ("__init__.py", "scenes.py"))
    if mutant is not None:
        fname, old, new = mutant
        path = os.path.join(work, "oracle", fname)
        src = open(path).read()
        assert src.count(old) == 1, f"mutation site not unique in {fname}: {old!r}"
        with open(path, "w") as f:
            f.write(src.replace(old, new))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", *(os.path.join("tests", s) for s in PIN_SUITES), "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"], cwd=work, env=env, capture_output=True,
                       text=True, timeout=900)
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else r.stderr[-500:]
    failed = int(m.group(1)) if (m := re.search(r"(\d+) failed", tail)) else 0
    passed = int(m.group(1)) if (m := re.search(r"(\d+) passed", tail)) else 0
    assert "error" not in tail, r.stdout[-3000:] + r.stderr[-2000:]
    return failed, passed, r.stdout


def test_unmutated_copy_passes_every_pin(tmp_path):
    failed, passed, out = run_pins(str(tmp_path))
    assert failed == 0 and passed >= 30, out[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    failed, passed, out = run_pins(str(tmp_path), MUTANTS[name])
    assert failed >= 1, f"mutant '{name}' passed every pin:\n{out[-2000:]}"
