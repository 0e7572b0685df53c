"""The pins catch plausible mistakes in the oracle. Each case plants one
mistake in a copy of oracle.c (a flipped operand order, a dropped factor, a
transposed index, a wrong constant), builds it, and runs the closed-form,
invariant and brute-force pins against it in a child process: at least one
must fail. The stored regression fixture of the oracle's own output is left
out, so that only pins fixed by the paper and the mathematics count."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "vertex normal operands swapped":
        ("d3 n = cross(sub(vb, va), sub(vc, va));", "d3 n = cross(sub(vc, va), sub(vb, va));"),
    "tie prefers the negative side":
        ("if ((t >= 0.0) != (best->t >= 0.0)) return t >= 0.0;", "if ((t >= 0.0) != (best->t >= 0.0)) return t < 0.0;"),
    "hit normal weights transposed":
        ("m = add(m, scl(ldd(j->hn, j->hf[3 * tri + k]), b[k]));",
         "m = add(m, scl(ldd(j->hn, j->hf[3 * tri + k]), b[(k + 1) % 3]));"),
    "bitangent handedness dropped":
        ("        d3 B = scl(cross(N, Tt), j->wsign[f]);\n        d3 nh = hit_normal(j, tri, hb);",
         "        d3 B = cross(N, Tt);\n        d3 nh = hit_normal(j, tri, hb);"),
    "ray direction not normalised":
        ("    d3 d = normalize(s);\n    double tol = 1e-5 * j->diam;", "    d3 d = s;\n    double tol = 1e-5 * j->diam;"),
    "displacement sign flipped":
        ("disp = h.tri >= 0 ? h.t : 0.0;", "disp = h.tri >= 0 ? -h.t : 0.0;"),
    "RGB8 scale 128":
        ("double r = v * 127.0;", "double r = v * 128.0;"),
    "dilated normal not renormalised":
        ("std3(nts, i, norm(mm) > 0 ? normalize(mm) : mk(0, 0, 1));", "std3(nts, i, mm);"),
    "tangent not made orthogonal to the normal":
        ("        d3 Tt = normalize(sub(ts, scl(N, dot(ts, N))));\n        d3 B = scl(cross(N, Tt), j->wsign[f]);\n        d3 nh",
         "        d3 Tt = normalize(ts);\n        d3 B = scl(cross(N, Tt), j->wsign[f]);\n        d3 nh"),
}

# the next rows' functions, each with the pins of its own row
ROW_MUTANTS = {
    "closest point: edge parameter not clamped above":
        ("        if (s > 1.0) s = 1.0;\n        d3 y = add(a, scl(e, s));", "        d3 y = add(a, scl(e, s));",
         ["tests/test_oracle_closest.py"]),
    "closest point: edge barycentrics swapped":
        ("b[k] = 1.0 - s; b[(k + 1) % 3] = s; b[(k + 2) % 3] = 0.0;",
         "b[k] = s; b[(k + 1) % 3] = 1.0 - s; b[(k + 2) % 3] = 0.0;", ["tests/test_oracle_closest.py"]),
    "QEM placement parameter measured from the far end":
        ("double t = dot(sub(x, v0), e) / ee;", "double t = dot(sub(x, v1), e) / ee;", ["tests/test_oracle_qem.py"]),
    "exterior fill gate dropped":
        ("if (dot(nf_, ldd(nrm, g)) > 0.0) { exterior[g] = 1; queue[qt++] = g; }",
         "{ exterior[g] = 1; queue[qt++] = g; }", ["tests/test_oracle_hidden.py"]),
    "loss: normal term averaged over every ray texel instead of the hit texels":
        ("    return (sum_t + lambda * sum_n) * inv;",
         "    int64_t nray = 0;\n    for (int64_t k = 0; k < ntex; ++k) nray += face[k] >= 0;\n"
         "    return sum_t * inv + lambda * sum_n / (double)nray;", ["tests/test_oracle_grad.py"]),
    "baked mean: map codes decoded about 127":
        ("d3 c = normalize(mk((q8[0] - 128.0) / 127.0, (q8[1] - 128.0) / 127.0, (q8[2] - 128.0) / 127.0));",
         "d3 c = normalize(mk((q8[0] - 127.0) / 127.0, (q8[1] - 127.0) / 127.0, (q8[2] - 127.0) / 127.0));",
         ["tests/test_oracle_map_error.py"]),
    "baked mean: texel row read from the far side":
        ("const uint8_t *q8 = m->rgba + 4 * ((int64_t)y * j->W + x);",
         "const uint8_t *q8 = m->rgba + 4 * ((int64_t)(j->H - 1 - y) * j->W + x);", ["tests/test_oracle_map_error.py"]),
    "baked mean: bitangent handedness dropped":
        ("    d3 B = scl(cross(N, Tt), j->wsign[f]);\n    int x = (int)floor(u * j->W)",
         "    d3 B = cross(N, Tt);\n    int x = (int)floor(u * j->W)", ["tests/test_oracle_map_error.py"]),
    "backprojection: a counted view within rounding of its decision never left out":
        ("vo[nvo].absent_ok = ak || !counted;", "vo[nvo].absent_ok = !counted;", ["tests/test_oracle_backproject.py"]),
    "backprojection incidence exponent dropped":
        ("L[nk] = log((double)weights[k]) + alpha * log(I);", "L[nk] = log((double)weights[k]) + log(I);",
         ["tests/test_oracle_backproject.py"]),
}

PINS = ["tests/test_oracle_bake.py", "tests/test_oracle_hit.py", "tests/test_oracle_raster.py",
        "tests/test_golden.py::test_encode_fixture", "tests/test_golden.py::test_dilation_fixture",
        "tests/test_golden.py::test_flat_plane_fixture"]


def _build_mutant(old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, "the mutation site moved"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", str(lib), str(mutant), "-lm", "-lpthread"])
    return lib


def _pins_fail(lib, pins):
    env = dict(os.environ, AG_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 1, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(ROW_MUTANTS))
def test_row_pins_catch_planted_mistake(name, tmp_path):
    old, new, pins = ROW_MUTANTS[name]
    failed, out = _pins_fail(_build_mutant(old, new, tmp_path), pins)
    assert failed, f"no pin caught '{name}':\n{out}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "the mutation site moved"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", str(lib), str(mutant), "-lm", "-lpthread"])
    env = dict(os.environ, AG_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"no pin caught '{name}':\n{r.stdout[-2000:]}"
