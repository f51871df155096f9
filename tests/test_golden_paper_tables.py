"""Checks against values printed in the paper (fixtures in tests/golden/paper_tables.txt).

* Table 1: the multiple-traces formulation has 8 dense operators and 4 unknown
  potentials -- the oracle's discrete MTF (Sec. 2.2, eq. mtf:discrete) must have
  exactly that structure: V, K, T, D on each grid, and 2 N_ext + 2 N_int unknowns.
* Table 2: the printed wavenumbers are 2 pi f / c of each medium (the plane wave of
  eq. planewave); this fixes the reading of Sec. 5.3, whose text repeats "k_ext" for
  what Table 2 lists as the interior wavenumber 5.7.
* Table 3: the nonconforming system couples N_ext + N_int = N_nodes vertices, so the
  MTF has 2 N_nodes unknowns, as the oracle's matrix does for any pair of grids.
"""
import math
import os

import numpy as np

import bem_inputs as bi

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(tag):
    out = []
    with open(os.path.join(HERE, "golden", "paper_tables.txt")) as fh:
        for line in fh:
            parts = line.split()
            if parts and parts[0] == tag:
                out.append(parts[1:])
    return out


def test_table1_mtf_has_8_operators_and_4_potentials():
    from oracle.mtf import mtf_blocks, mtf_matrix, solve_transmission
    row = [r for r in _rows("table1") if r[0] == "multiple-traces"][0]
    n_ops, n_pot = int(row[2]), int(row[3])
    ve, te, vi, ti = bi.transmission_pair(1, 1, seed=5)
    B = mtf_blocks(ve, te, vi, ti, 1.0, 2.0)
    dense = [B["ext"][k] for k in ("V", "K", "T", "D")] + [B["int"][k] for k in ("V", "K", "T", "D")]
    assert len(dense) == n_ops
    assert all(np.count_nonzero(np.abs(A) > 0) > 0.9 * A.size for A in dense)  # dense blocks
    out = solve_transmission(ve, te, vi, ti, 1.0, 2.0, 1.0, np.array([0.0, 0.0, 1.0]), blocks=B)
    pots = [out[k] for k in ("v_ext", "w_ext", "v_int", "w_int")]
    assert len(pots) == n_pot
    assert mtf_matrix(B, 1.0).shape == (2 * len(ve) + 2 * len(vi),) * 2


def test_table2_wavenumbers_are_two_pi_f_over_c():
    for name, f, ce, ci, _re, _ri, ke, ki in _rows("table2"):
        f, ce, ci, ke, ki = map(float, (f, ce, ci, ke, ki))
        assert abs(2 * math.pi * f / ce - ke) < 0.05, name
        assert abs(2 * math.pi * f / ci - ki) < 0.05, name


def test_table3_node_counts_set_the_system_size():
    from oracle.mtf import mtf_blocks, mtf_matrix
    for name, ne, nic, nnc, nin, nnn in _rows("table3"):
        ne, nic, nnc, nin, nnn = map(int, (ne, nic, nnc, nin, nnn))
        assert ne + nic == nnc and ne + nin == nnn, name
    ve, te, vi, ti = bi.transmission_pair(1, 0, seed=7)
    B = mtf_blocks(ve, te, vi, ti, 1.0, 1.5)
    assert mtf_matrix(B, 2.0).shape[0] == 2 * (len(ve) + len(vi))


def test_cube_benchmarks_follow_tables_2_and_3():
    """The unit-cube benchmarks timed by bench.py use Table 2's physics (f, c, rho of
    both media) and nonconforming cube grids whose node counts are within 10 % of
    Table 3's N_ext and nonconforming N_int."""
    import bench
    t2 = {r[0]: list(map(float, r[1:6])) for r in _rows("table2")}
    t3 = {r[0]: (int(r[1]), int(r[4])) for r in _rows("table3")}
    for b in bench.CUBE_BENCHMARKS:
        key = b["name"].replace(" ", "-")
        assert [b["f"], b["c_ext"], b["c_int"], b["rho_ext"], b["rho_int"]] == t2[key], key
        assert (b["N_ext"], b["N_int"]) == t3[key], key
        for N in t3[key]:
            n = bench.cube_edge_nodes(N)
            assert abs(6 * n * n + 2 - N) <= 0.1 * N, (key, N, n)
