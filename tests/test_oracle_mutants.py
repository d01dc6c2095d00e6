"""Planted mistakes in the oracle must be caught by its pins (no GPU).

Each mutant is a copy of ``oracle/rfps_oracle.c`` with one plausible mistake
(a dropped term, a wrong sign or index, a transposed operand, a wrong tie or
pruning rule), compiled into a temporary library.  The pins of ``pins.py``
run against it; at least one of them has to fail.
"""

import os
import shutil
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "rfps_oracle.c")

# (name, text to find, replacement) -- the first occurrence is replaced
MUTANTS = [
    ("drop_dz_term", "    return s + zz;", "    return s;"),
    ("wrong_sign", "float dx = p[0] - q[0];", "float dx = p[0] + q[0];"),
    ("transposed_operand", "float dy = p[1] - q[1];", "float dy = p[1] - q[2];"),
    ("ties_to_largest_index", "if (D[i] > best_v) {      /* strict", "if (D[i] >= best_v) {      /* strict"),
    ("init_zero_not_inf", "        D[i] = INFINITY;\n    out[0] = start;", "        D[i] = 0.0f;\n    out[0] = start;"),
    ("max_instead_of_min", "                if (d < D[i])\n                    D[i] = d;\n                if (D[i] > best_v)",
     "                if (d > D[i])\n                    D[i] = d;\n                if (D[i] > best_v)"),
    ("round_not_floor", "float f = floorf(q);", "float f = roundf(q);"),
    ("wrong_alpha", "1.0f + 0.0009765625f", "1.0f + 0.01f"),
    ("voxel_id_axes_swapped", "(vz * (uint32_t)n_vox + vy) * (uint32_t)n_vox + vx",
     "(vx * (uint32_t)n_vox + vy) * (uint32_t)n_vox + vz"),
    ("centroid_only_pruning", "double lb = dc * margin_lo - rad[k] * (1.0 + ldexp(1.0, -48));",
     "double lb = dc;"),
    ("unsquared_skip_term", "xx >= D[i] || yy >= D[i] || zz >= D[i]", "xx >= D[i] || yy >= D[i] || dz >= D[i]"),
    ("voxel_ties_by_voxel_order", "(dv[k] == dv[kb] && dv_idx[k] < dv_idx[kb])", "(0)"),
]

PINS = [pins.pin_golden_fps, pins.pin_voxelize, pins.pin_closed_form, pins.pin_bruteforce,
        pins.pin_invariants, pins.pin_radiusfps_identity]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,find,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, find, repl):
    src = open(SRC).read()
    assert find in src, f"mutation site for {name} not found"
    mutated = src.replace(find, repl, 1)
    csrc = tmp_path / f"mut_{name}.c"
    csrc.write_text(mutated)
    so = tmp_path / f"libmut_{name}.so"
    oracle.build(str(csrc), str(so))
    lib = oracle.load(str(so))
    caught = []
    for pin in PINS:
        try:
            pin(lib)
        except (AssertionError, oracle.OracleError) as e:  # a pin disagreed
            caught.append((pin.__name__, repr(e)[:120]))
            break
    assert caught, f"no pin caught mutant {name}"


def test_unmutated_copy_passes(tmp_path):
    """Control: the same build route with no mutation passes every pin."""
    csrc = tmp_path / "copy.c"
    csrc.write_text(open(SRC).read())
    so = tmp_path / "libcopy.so"
    oracle.build(str(csrc), str(so))
    lib = oracle.load(str(so))
    for pin in PINS:
        pin(lib)
