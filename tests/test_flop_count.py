"""The algorithmic operation counts behind the benchmark's roofline figures
are those of the oracle's own source: oracle/flopcount.cpp compiles
w5ct_oracle.c with a counting scalar type, and this test builds it, runs it
for WENO-JS and WENO-Z and checks the constants bench.py divides by kernel
times (per cell and per interface of one sweep, Sec. 2.2 and Appendix A;
the CT transport fluxes of Eqs. fct1-fct6; per zone of a whole RK4 + CT
step, Secs. 2.1 and 2.3)."""
import json
import os
import subprocess

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def counts(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("flopcount") / "flopcount")
    src = os.path.join(ROOT, "oracle", "flopcount.cpp")
    subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-o", exe, src, "-lm"], check=True)
    out = {}
    for variant in (0, 1):
        r = subprocess.run([exe, str(variant)], check=True, capture_output=True, text=True)
        out[variant] = json.loads(r.stdout)
    return out


@pytest.mark.parametrize("variant", [0, 1])
def test_bench_flop_constants_equal_the_oracle_counts(counts, variant):
    c = counts[variant]
    assert c["cell"] == bench.CELL_FLOPS
    assert c["face_core"] == bench.FACE_FLOPS[variant]
    # a whole sweep = cells + faces + transport fluxes + the divergence (15)
    assert c["face"] == bench.FACE_FLOPS[variant] + bench.CT_FLUX_FLOPS
    assert c["sweep"] == bench.SWEEP_FLOPS_PER_ZONE[variant] + c["div"]
    assert round(c["step"]) == bench.STEP_FLOPS_PER_ZONE[variant]
    assert abs(c["step"] - round(c["step"])) < 0.01
    assert round(c["adjoint_step"]) == bench.ADJOINT_STEP_FLOPS_PER_ZONE[variant]


def test_reverse_mode_count_is_a_few_forward_counts(counts):
    """The reverse sweep of a step costs between one and four times its
    forward operations (the bound of reverse-mode differentiation for
    +, -, * and /: at most two multiplications and two additions per
    operand contribution)."""
    for variant in (0, 1):
        c = counts[variant]
        assert c["step"] < c["step_reverse"] < 4 * c["step"], (variant, c)
        assert c["adjoint_step"] == pytest.approx(c["step"] + c["step_reverse"])


def test_step_count_is_four_stages_of_three_sweeps_plus_ct(counts):
    """The step is four stages of three sweeps; the rest (cell-field
    interpolation, stage update, EMFs, face updates) is a small remainder."""
    for variant in (0, 1):
        c = counts[variant]
        rest = c["step"] - 12 * c["sweep"]
        assert 0 < rest < 0.02 * c["step"], (variant, rest)
