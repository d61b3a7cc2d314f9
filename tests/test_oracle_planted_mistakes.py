"""The oracle's pins have teeth: each plausible mistake below is planted in a
scratch copy of the oracle (on the CPU), the copy is built, and the pins
that cover that part of the method are run against it; at least one must
fail.  The real oracle is never modified.

Each case is (what the mistake is, the exact source line(s), the mistaken
line(s), the pytest -k expression selecting the pins of that part)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    ("Nyquist bin by exp(-i pi d) instead of cos(pi d) (R3)",
     "    if (2 * k == M) return cos(ORACLE_PI * d);",
     "    if (2 * k == M) return cos(ORACLE_PI * d) - I * sin(ORACLE_PI * d);",
     "shift or gibbs"),
    ("shift phasor sign (R1)",
     "    double ang = -2.0 * ORACLE_PI * (double)ks * d / (double)M;",
     "    double ang = 2.0 * ORACLE_PI * (double)ks * d / (double)M;",
     "shift"),
    ("y-shear sign of the rotation (R6)",
     "    double m2 = shear_pass(P, M, 1, s);",
     "    double m2 = shear_pass(P, M, 1, -s);",
     "rotat or shear"),
    ("even median: the lower middle value (R15, FP32)",
     "    float s = v[n / 2 - 1] + v[n / 2];\n    return s * 0.5f;",
     "    float s = v[n / 2 - 1] + v[n / 2 - 1];\n    return s * 0.5f;",
     "median or collapse"),
    ("even median: the lower middle value (R15, FP64)",
     "    return (v[n / 2 - 1] + v[n / 2]) * 0.5;",
     "    return (v[n / 2 - 1] + v[n / 2 - 1]) * 0.5;",
     "median or collapse or adi or reduce"),
    ("angle gate not strict (R11)",
     "        mask[k] = in_time && fabs(parang[k] - parang[i]) > amin;",
     "        mask[k] = in_time && fabs(parang[k] - parang[i]) >= amin;",
     "gate"),
    ("annulus includes its outer edge (R12)",
     "        if (edges[a] * edges[a] <= rho2 && rho2 < edges[a + 1] * edges[a + 1]) return a;",
     "        if (edges[a] * edges[a] <= rho2 && rho2 <= edges[a + 1] * edges[a + 1]) return a;",
     "adi"),
    ("time gate not strict (R19)",
     "        int in_time = times == NULL || fabs(times[k] - times[i]) < t_max;",
     "        int in_time = times == NULL || fabs(times[k] - times[i]) <= t_max;",
     "time_gate"),
    ("sky tie takes the later sky (R23)",
     "            if (fabs(sky_times[s] - frame_times[t]) < fabs(sky_times[j] - frame_times[t])) j = s;",
     "            if (fabs(sky_times[s] - frame_times[t]) <= fabs(sky_times[j] - frame_times[t])) j = s;",
     "sky"),
    ("bad pixel map not strict (R24)",
     "    for (size_t p = 0; p < NN; p++) map[p] = fabs((double)ref[p] - (double)med) > C * sigma;",
     "    for (size_t p = 0; p < NN; p++) map[p] = fabs((double)ref[p] - (double)med) >= C * sigma;",
     "bad_pixel"),
    ("centroid seed threshold not strict (R26)",
     "    if (!((double)f[best] > thresh)) return 0;",
     "    if (!((double)f[best] >= thresh)) return 0;",
     "centroid"),
    ("patch grown with 4-connectivity (R26)",
     "                if ((!dr && !dc) || rr < 0 || rr >= H || cc < 0 || cc >= W) continue;",
     "                if ((!dr && !dc) || (dr && dc) || rr < 0 || rr >= H || cc < 0 || cc >= W) continue;",
     "centroid"),
    ("Moffat dI/dx0 sign (R28)",
     "        grad[1] = A * be * Pu * 2.0 * dx / (al * al);",
     "        grad[1] = -A * be * Pu * 2.0 * dx / (al * al);",
     "moffat"),
    ("injection angle pa0 - parang (R31)",
     "            double ang = (pa0[j] + parang[t]) * ORACLE_PI / 180.0;",
     "            double ang = (pa0[j] - parang[t]) * ORACLE_PI / 180.0;",
     "inject"),
    ("bad pixel pass reads this pass's fills (R25)",
     "                            float w = g[(size_t)ii * N + jj];",
     "                            float w = f[(size_t)ii * N + jj];",
     "bad_pixel"),
    ("star mask includes its rim (R22)",
     "                if (ddx * ddx + ddy * ddy < mask_r * mask_r) continue;",
     "                if (ddx * ddx + ddy * ddy <= mask_r * mask_r) continue;",
     "sky"),
    ("aperture boundary strict (R33)",
     "                if (dx * dx + dy * dy <= radius * radius) s += (double)img[(size_t)row * N + col];",
     "                if (dx * dx + dy * dy < radius * radius) s += (double)img[(size_t)row * N + col];",
     "aperture"),
]


@pytest.mark.parametrize("name,old,new,kexpr", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, kexpr):
    mut = tmp_path / "mut"
    shutil.copytree(os.path.join(ROOT, "oracle"), mut / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    src_path = mut / "oracle" / "graphic_oracle.c"
    src = src_path.read_text()
    assert src.count(old) >= 1, f"the line to mutate is gone: {name}"
    src_path.write_text(src.replace(old, new))
    (mut / "tests").mkdir()
    for f in ("test_oracle_pins.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), mut / "tests" / f)
    if os.path.isdir(os.path.join(ROOT, "tests", "golden")):
        shutil.copytree(os.path.join(ROOT, "tests", "golden"), mut / "tests" / "golden")
    env = dict(os.environ, PYTHONPATH=f"{mut}{os.pathsep}{ROOT}")
    build = subprocess.run([sys.executable, "-c",
                            f"import oracle; assert oracle.__file__.startswith({str(mut)!r}); oracle.build(force=True)"],
                           cwd=mut, env=env, capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-p", "no:cacheprovider",
                          "-k", kexpr, "--rootdir", str(mut)], cwd=mut, env=env, capture_output=True, text=True)
    summary = [ln for ln in run.stdout.splitlines() if " passed" in ln or " failed" in ln or "error" in ln]
    assert run.returncode != 0 and any("failed" in ln for ln in summary), \
        f"no pin caught: {name}\n" + "\n".join(summary[-3:])
