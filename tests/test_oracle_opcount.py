"""The oracle's operation counter (oracle/opcount.cpp), which fixes the
algorithmic FP64 work per cell that the bench's roofline of the FP64 property
path divides by: its short forms reproduce the oracle's results, its
counting rules do what they say, and the bench uses the committed count."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import count_ops
from paper_2312_04830_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def counts():
    T, p, Y = W.flame_vortex_field(32)
    idx = np.linspace(0, T.size - 1, 4096).astype(np.int64)
    return oracle.op_counts(W.species_table(), T[idx], p[idx], Y[:, idx])


def test_short_forms_reproduce_the_oracle(counts):
    # factorised mixing and Chung sums, closed-form roots, species terms, ideal-gas sums
    assert counts["cells"] > 4000
    assert max(counts["check"]) < 1e-11, counts["check"]


def test_counting_rules():
    T, p, Y = W.uniform_cells(1024, seed=8)      # every species present in every cell
    c = oracle.op_counts(W.species_table(), T, p, Y)
    st, sh = c["steps"], c["short"]
    N = 9
    # mixing: the oracle's double sum is quadratic in N, the factorised form linear
    assert st["mixing"]["mul"] > 20 * N and sh["mixing"]["mul"] <= 5 * N
    # table set-up is not per-cell work: the composition takes N divisions by
    # the state-dependent sum (the divisions by W_k are multiplications)
    assert st["composition"]["div"] == pytest.approx(N)
    # one sqrt(T) per cell in the short species terms, whatever N
    assert sh["species_terms"]["sqrt"] == pytest.approx(1.0)
    # diagnostics are counted apart and not in the work
    assert "diagnostics" in st
    # Chung's dense correlation: Neufeld's three terms (a power and two
    # exponentials), the G2 and H2 exponentials and expm1 terms, the eta**
    # exponential and Vc^(2/3)
    assert st["Chung dense correlation"]["exp"] == pytest.approx(5.0)
    assert st["Chung dense correlation"]["expm1"] == pytest.approx(2.0)
    assert st["Chung dense correlation"]["pow"] == pytest.approx(2.0)


def test_counts_scale_with_species():
    """A one-species table against the 9-species one: the factorised sums shrink
    in proportion, the per-cell correlation work does not change."""
    T, p, Y = W.uniform_cells(512, seed=9)
    one = W.SpeciesTable(("O2",))
    c1 = oracle.op_counts(one, T, p, np.ones((1, T.size)))
    c9 = oracle.op_counts(W.species_table(), T, p, Y)
    # four products per species (x_k sqrt(a_k), its two derivatives, x_k b_k) and
    # the same few to close the sums
    per9, per1 = c9["short"]["mixing"]["mul"], c1["short"]["mixing"]["mul"]
    assert per9 - per1 == pytest.approx(8 * 4)
    assert c9["steps"]["Chung dense correlation"]["exp"] == c1["steps"]["Chung dense correlation"]["exp"]


def test_bench_uses_the_committed_count():
    with open(os.path.join(ROOT, "oracle", "op_counts_flame_vortex_256.json")) as f:
        rep = json.load(f)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.ALGO_FP64_FLOPS_PER_CELL["props_fp64"] == pytest.approx(rep["fp64_flops_per_cell"], rel=1e-9)
    # the committed record is what the script computes (a smaller sample agrees to 1 %)
    small = count_ops.count(grid=256, sample=8192)
    assert small["fp64_flops_per_cell"] == pytest.approx(rep["fp64_flops_per_cell"], rel=1e-2)
