"""Pins of the oracle's coupled (multi-cell) system: the paper's Multi-cells
integration of a group of cells as one ODE system.

The oracle writes a group as one mechanism over all its species.  Pinned
against things other than itself: the group's f is the cells' f side by side
(the system is block diagonal), and G identical copies of a cell integrate to
that cell's own solution with its own step sequence (the group norm of equal
parts is the cell's norm).
"""
import numpy as np

from paper_2501_00011_gb300 import synth


def test_group_derivative_is_block_diagonal(oracle_lib):
    m = synth.mechanism_small()
    cells = synth.random_cells(m.n_species, 3, T_range=(220, 310), P_range=(2e4, 1e5), seed=31)
    big = oracle_lib.replicate(m, 3)
    kt = np.concatenate([oracle_lib.rate_constants(m, cells.T[c], cells.P[c]) for c in range(3)])
    y = np.concatenate([cells.y[:, c] for c in range(3)])
    f = oracle_lib.deriv(big, kt, y)
    for c in range(3):
        fc = oracle_lib.deriv(m, kt[c * m.n_reactions:(c + 1) * m.n_reactions], cells.y[:, c])
        assert np.array_equal(f[c * m.n_species:(c + 1) * m.n_species], fc)
    J = oracle_lib.jacobian(big, kt, y)
    S = m.n_species
    for a in range(3):
        for b in range(3):
            if a != b:
                assert not np.any(J[a * S:(a + 1) * S, b * S:(b + 1) * S])


def test_identical_copies_reproduce_the_single_cell(oracle_lib):
    for mk, rtol, atol in ((synth.mechanism_small, 1e-6, 1e-14), (synth.mechanism_tropo, 1e-4, 1e-10)):
        m = mk()
        one = synth.random_cells(m.n_species, 1, T_range=(230, 300), P_range=(3e4, 1e5), seed=32)
        group = synth.subset(one, [0, 0, 0, 0])
        y1, s1 = oracle_lib.solve_cells(m, one, 600.0, rtol, atol)
        yg, sg = oracle_lib.solve_coupled(m, group, 600.0, rtol, atol, 4)
        assert sg["status"][0] == 0 and s1["status"][0] == 0
        assert sg["steps"][0] == s1["steps"][0] and sg["newton_iters"][0] == s1["newton_iters"][0]
        mask = np.abs(y1[:, 0]) > 1e-20
        for c in range(4):
            assert np.all(np.abs(yg[mask, c] - y1[mask, 0]) <= 1e-10 * np.abs(y1[mask, 0]))
