"""Mutation check of the oracle's pins (test infrastructure).

Each mutation plants one plausible mistake (a dropped factor, a wrong sign, a
wrong index, a missing term) in a copy of the oracle's C sources, builds that
copy into a temporary library and runs the pin tests against it (through the
ORACLE_LIB variable that ``oracle.lib`` honours); a pin set is good when every
mutant makes at least one of its tests fail.  The sources beside this file
are never modified.

    python -m oracle.mutation_check            # every mutant, a table, exit 1 if one survives
    python -m oracle.mutation_check t_sign      # selected mutants
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_step.py"]
_SHOCK = ["tests/test_oracle_shock.py"]
_ADJ = ["tests/test_oracle_adjoint.py"]
_C = "pic_oracle.c"
_CA = "pic_oracle_adj.c"

# (name, source file, original text, mutated text, pin tests)
MUTATIONS = [
    ("half_kick_dropped", _C, "u1[a] = c * u[a] + 0.5 * qm * e[a];\n  const double g1",
     "u1[a] = c * u[a] + qm * e[a];\n  const double g1", _PINS),
    ("t_sign", _C, "t[a] = qm * b[a] / (2.0 * c * g1)", "t[a] = -qm * b[a] / (2.0 * c * g1)", _PINS),
    ("gamma1_missing", _C, "t[a] = qm * b[a] / (2.0 * c * g1)", "t[a] = qm * b[a] / (2.0 * c)", _PINS),
    ("by_stagger", _C, "{0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}", "{0.0, 0.5, 0.5}, {0.5, 0.5, 0.0}", _PINS),
    ("curl_b_sign", _C, "F[EX * P + p] += g->c * cx;", "F[EX * P + p] -= g->c * cx;", _PINS),
    ("curl_e_cz_swapped", _C,
     "const double cz = dplus_o(g, F, EY, 0, i, j, k) - dplus_o(g, F, EX, 1, i, j, k);",
     "const double cz = dplus_o(g, F, EX, 1, i, j, k) - dplus_o(g, F, EY, 0, i, j, k);", _PINS),
    ("filter_weights", _C, "0.5 * tmp[at(g, i, j, k)]", "0.4 * tmp[at(g, i, j, k)]", _PINS),
    ("w2_uses_i1", _C, "W2[d] = 0.5 * (x2[d] + xr[d]) - (double)i2[d];",
     "W2[d] = 0.5 * (x2[d] + xr[d]) - (double)i1[d];", _PINS),
    ("relay_min_max", _C, "xr[d] = fmin(lo, fmax(hi, 0.5 * (x1[d] + x2[d])));",
     "xr[d] = fmax(lo, fmin(hi, 0.5 * (x1[d] + x2[d])));", _PINS),
    ("segment_term_sign", _C, "(o[b] == o[c] ? 1.0 : -1.0)", "(o[b] == o[c] ? -1.0 : 1.0)", _PINS),
    ("abs_term_dropped", _C, "+= g_abs ? fabs(v) : v;", "+= v;", _PINS),
    ("move_without_c", _C, "dx[d * n + p] = g->c * up[d] / gam;", "dx[d * n + p] = up[d] / gam;", _PINS),
    ("e_minus_j_sign", _C, "F[(EX + a) * P + p] -= F[(JX + a) * P + p];",
     "F[(EX + a) * P + p] += F[(JX + a) * P + p];", _PINS),
    ("rho_weight", _C,
     "              wt *= o[d] ? w[d] : 1.0 - w[d];\n            }\n          }\n          if (!skip)",
     "              wt *= o[d] ? 1.0 - w[d] : w[d];\n            }\n          }\n          if (!skip)",
     _PINS),
    ("gather_weight", _C,
     "              wt *= o[d] ? w[d] : 1.0 - w[d];\n            }\n          }\n          if (skip)",
     "              wt *= o[d] ? w[d] : w[d];\n            }\n          }\n          if (skip)", _PINS),
    ("wall_no_split", _C, "    if (g_wall > 0 && x2[0] < (double)g_wall) {\n      const double w",
     "    if (0 && x2[0] < (double)g_wall) {\n      const double w", _SHOCK),
    ("wall_crossing_point", _C, "xc[d] = x1[d] + s * (x2[d] - x1[d]);", "xc[d] = x1[d];", _SHOCK),
    ("ey_image_sign", _C, "F[EY * P + a] = -F[EY * P + ri];", "F[EY * P + a] = F[EY * P + ri];", _SHOCK),
    ("bz_image_index", _C, "F[BZ * P + a] = F[BZ * P + rh];", "F[BZ * P + a] = F[BZ * P + ri];", _SHOCK),
    ("inject_time", _C, "v_up * (double)(s + 1);", "v_up * (double)s;", _SHOCK),
    ("front_without_upstream", _C, "return (X - x0) + v_up * (double)s;", "return (X - x0);", _SHOCK),
    ("no_u_flip", _C, "        u[p] = -u[p];\n", "\n", _SHOCK),
    ("no_tangential_e_zero", _C, "      F[EY * P + at(g, w, j, k)] = 0.0;\n", "\n", _SHOCK),
    ("mirror_end", _C, "xm[0] = 2.0 * w - x2[0];", "xm[0] = x2[0];", _SHOCK),
    ("adj_mid_branch", _CA, "        x1b[d] += 0.5 * xrb;\n        x2b[d] += 0.5 * xrb;",
     "        x1b[d] += 0.0 * xrb;\n        x2b[d] += 0.5 * xrb;", _ADJ),
    ("adj_segment_term", _CA, "        Dbar[bb] += Fl * jb * sgn * Ds[cc] / 12.0;",
     "        Dbar[bb] += 0.0;", _ADJ),
    ("adj_curl_direction", _CA, "  add_curl(g, A, BX, 0, -0.5 * g->c, d);",
     "  add_curl(g, A, BX, 1, -0.5 * g->c, d);", _ADJ),
    ("adj_boris_cross", _CA, "  crossa(u3b, v, tmp);", "  crossa(v, u3b, tmp);", _ADJ),
    ("adj_gamma_term", _CA,
     "  for (int a = 0; a < 3; ++a) u1b[a] += -g1b * g1 * g1 * g1 * u1[a] / (c * c);", "", _ADJ),
    ("adj_move_projection", _CA, "u2b[a] += c / gam * (dnb[a] - u2[a] * ud / (gam * gam));",
     "u2b[a] += c / gam * dnb[a];", _ADJ),
    ("adj_gather_position", _CA,
     "      for (int d = 0; d < g->dim; ++d) xbar[d] += corner_weight(g, w, o, -1, d) * f * vbar;",
     "", _ADJ),
]


def _build(tmp: str, fname: str, before: str, after: str) -> str:
    for f in (_C, _CA, "pic_oracle.h"):
        shutil.copy(os.path.join(_HERE, f), os.path.join(tmp, f))
    path = os.path.join(tmp, fname)
    src = open(path).read()
    if src.count(before) != 1:
        raise RuntimeError(f"mutation site not found exactly once in {fname}: {before[:60]!r}")
    open(path, "w").write(src.replace(before, after))
    out = os.path.join(tmp, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", os.path.join(tmp, _C), os.path.join(tmp, _CA),
                           "-o", out, "-lm"])
    return out


def run_one(name: str) -> tuple[bool, str]:
    """Build mutant `name` and run its pins; returns (caught, last pytest line)."""
    (_, fname, before, after, tests), = [m for m in MUTATIONS if m[0] == name]
    with tempfile.TemporaryDirectory() as tmp:
        libpath = _build(tmp, fname, before, after)
        env = dict(os.environ, ORACLE_LIB=libpath)
        r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-x", "-q", "-m", "not gpu",
                            "-p", "no:cacheprovider"], cwd=_ROOT, env=env, capture_output=True,
                           text=True)
    lines = r.stdout.strip().splitlines()
    return r.returncode != 0, lines[-1] if lines else r.stderr.strip()[-200:]


def main(argv: list[str]) -> int:
    names = argv or [m[0] for m in MUTATIONS]
    survivors = []
    for name in names:
        caught, last = run_one(name)
        print(f"{name:24s} {'caught' if caught else 'SURVIVED'}  {last}", flush=True)
        if not caught:
            survivors.append(name)
    print(f"{len(names) - len(survivors)} of {len(names)} mutants caught")
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
