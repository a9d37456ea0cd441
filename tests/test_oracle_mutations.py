"""The oracle's pins catch plausible mistakes: each test plants one mistake in a copy of the
oracle's C source (a wrong sign, a wrong index, a wrong factor, swapped operands), builds that
copy, and checks that at least one of the pins in tests/test_oracle_pins.py fails against it.
Nothing here touches the oracle itself: the mutant is compiled to a temporary library and the
oracle module is pointed at it for the duration of one test.
"""
import math
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sgeo_oracle.c")

# (name, original text, mutated text, pins expected to notice)
MUTATIONS = [
    ("unfold sign across an edge",
     "x[i] = a * U->e[i] - c * U->uf2[i];", "x[i] = a * U->e[i] + c * U->uf2[i];",
     [lambda: pins.test_folded_strip_matches_development([(4, 0.7)]),
      lambda: pins.test_polycube_exact_face_sequences([(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)])]),
    ("straightest rule splits theta unevenly",
     "double half = 0.5 * m->theta[v0];", "double half = 0.45 * m->theta[v0];",
     [lambda: pins.test_cone_vertex_straightest_rule(1.3 * math.pi), pins.test_cube_worked_examples]),
    ("exit parameter divides by the wrong edge's rate",
     "double ti = fmax(s->b[i], 0.0) / (-bd[i]);", "double ti = fmax(s->b[i], 0.0) / (-bd[(i + 1) % 3]);",
     [pins.test_flat_mesh_endpoint_is_p_plus_v, pins.test_cube_worked_examples]),
    ("carried vector mirrored at a vertex",
     "w[3 * q + i] = wl[q] * (cos(phi[q]) * dout[i] + sin(phi[q]) * c[i]);",
     "w[3 * q + i] = wl[q] * (cos(phi[q]) * dout[i] - sin(phi[q]) * c[i]);",
     [lambda: pins.test_cone_vertex_straightest_rule(1.8 * math.pi)]),
    ("carried vector mirrored at a vertex, against the development at a vertex of angle sum 2pi",
     "w[3 * q + i] = wl[q] * (cos(phi[q]) * dout[i] + sin(phi[q]) * c[i]);",
     "w[3 * q + i] = wl[q] * (cos(phi[q]) * dout[i] - sin(phi[q]) * c[i]);",
     [lambda: pins.test_vertex_on_a_fold_matches_development(0.9)]),
    ("straightest rule splits theta unevenly, against the development at a vertex of angle sum 2pi",
     "double half = 0.5 * m->theta[v0];", "double half = 0.45 * m->theta[v0];",
     [lambda: pins.test_vertex_on_a_fold_matches_development(-1.7)]),
    ("barycentrics swapped on entering the neighbour",
     "s->b[gj] = sj; s->b[gk] = sk; s->b[gz] = 0.0;", "s->b[gj] = sk; s->b[gk] = sj; s->b[gz] = 0.0;",
     [pins.test_flat_mesh_endpoint_is_p_plus_v,
      lambda: pins.test_polycube_exact_face_sequences([(0, 0, 0)])]),
    ("corner angles summed with a wrong factor",
     "m->theta[v] += vangle(a, b);", "m->theta[v] += 1.001 * vangle(a, b);",
     [pins.test_vertex_angle_sums_gauss_bonnet, lambda: pins.test_cone_vertex_straightest_rule(2.4 * math.pi)]),
    ("GFD position columns along swapped frame axes",
     "vcopy(step, c == 0 ? eu : ev); vscale(step, eps_p);", "vcopy(step, c == 0 ? ev : eu); vscale(step, eps_p);",
     [pins.test_ep_and_gfd_match_central_differences, pins.test_flat_gradients_closed_form]),
    ("hole avoidance slides the wrong way along the hit edge",
     "const int tgt = de >= 0.0 ? k2 : j;", "const int tgt = de < 0.0 ? k2 : j;",
     [pins.test_hole_avoidance_closed_forms_on_a_square_with_a_hole]),
    ("hole avoidance turns back along the boundary",
     "k = bvert[0] == came_from ? 1 : 0;", "k = bvert[0] == came_from ? 0 : 1;",
     [pins.test_hole_avoidance_closed_forms_on_a_square_with_a_hole]),
    ("EP gradient with its two columns transposed",
     "grad_v[3 * i + k] = gp * ep[k] + gq * eq[k];", "grad_v[3 * i + k] = gq * ep[k] + gp * eq[k];",
     [pins.test_ep_and_gfd_match_central_differences, pins.test_flat_gradients_closed_form]),
]


def _build_mutant(text: str, tmp: str) -> str:
    src = os.path.join(tmp, "mutant.c")
    with open(src, "w") as f:
        f.write(text)
    out = os.path.join(tmp, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", out, src, "-lm"])
    return out


@pytest.mark.parametrize("name,orig,mut,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_a_planted_mistake(name, orig, mut, checks):
    text = open(SRC).read()
    assert text.count(orig) == 1, f"mutation site not found: {orig}"
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    saved_out, saved_lib = oracle._OUT, oracle._lib
    try:
        path = _build_mutant(text.replace(orig, mut), tmp)
        oracle._OUT, oracle._lib = path, None
        caught = []
        for check in checks:
            try:
                check()
            except (AssertionError, ValueError, IndexError, FloatingPointError):
                caught.append(check)
        assert caught, f"no pin noticed the planted mistake: {name}"
    finally:
        oracle._OUT, oracle._lib = saved_out, saved_lib
        shutil.rmtree(tmp, ignore_errors=True)


def test_unmutated_copy_passes_the_same_pins():
    """Control: the same procedure with no mutation passes every pin used above."""
    tmp = tempfile.mkdtemp(prefix="oracle_copy_")
    saved_out, saved_lib = oracle._OUT, oracle._lib
    try:
        oracle._OUT, oracle._lib = _build_mutant(open(SRC).read(), tmp), None
        seen = set()
        for _, _, _, checks in MUTATIONS:
            for check in checks:
                if id(check) not in seen:
                    seen.add(id(check))
                    check()
    finally:
        oracle._OUT, oracle._lib = saved_out, saved_lib
        shutil.rmtree(tmp, ignore_errors=True)
