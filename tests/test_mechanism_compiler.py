"""The host-side mechanism compiler (a2-a5 programs), replayed on the CPU.

The compiler's warp programs are replayed in numpy (program_emulator) on
seeded states and checked against the oracle and numpy: the f program
against the oracle's f, the M / LU / forward / backward programs against a
dense solve of (I - c J) with the oracle's J, the transposed solves against
the transposed dense solve, and the adjoint's J^T mu program against J^T mu.
The replay also checks every pass for read/write conflicts and every slot
for bounds, and the symbolic fill against an elimination of the Jacobian
pattern written out here from the reaction tables.
"""
import numpy as np
import pytest

import program_emulator as pe
from paper_2501_00011_gb300 import synth

MECHS = {"small": synth.mechanism_small, "tropo": synth.mechanism_tropo, "pressure": synth.mechanism_tropo_pressure,
         # two register-slot sizes the named workloads do not reach: 33-64 and 97-128 (the maximum) species
         "s50": lambda: synth.random_mechanism(50, 130, 40, 13, name="synthetic_50sp_130rx"),
         "s128": lambda: synth.random_mechanism(128, 330, 100, 34, name="synthetic_128sp_330rx")}


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    return pe.build_dumper(str(tmp_path_factory.mktemp("progdump")))


@pytest.fixture(scope="module")
def compiled(dumper, tmp_path_factory):
    wd = str(tmp_path_factory.mktemp("programs"))
    return {k: (mk(), pe.Compiled(dumper, mk(), wd)) for k, mk in MECHS.items()}


def jacobian_pattern(m):
    S = m.n_species
    P = np.eye(S, dtype=bool)
    for j in range(m.n_reactions):
        nu = {}
        for s in m.reac[j, :m.n_reac[j]]:
            nu[int(s)] = nu.get(int(s), 0.0) - 1.0
        for p, yv in zip(m.prod[j, :m.n_prod[j]], m.yld[j, :m.n_prod[j]]):
            nu[int(p)] = nu.get(int(p), 0.0) + float(yv)
        for l in set(int(s) for s in m.reac[j, :m.n_reac[j]]):
            for i, v in nu.items():
                if v != 0.0:
                    P[i, l] = True
    return P


@pytest.mark.parametrize("name", list(MECHS))
def test_symbolic_fill_is_the_elimination_of_the_pattern(compiled, name):
    m, cp = compiled[name]
    P = jacobian_pattern(m)
    assert cp.nnz_jac == int(P.sum())
    order = np.argsort(cp.pos)                      # species at each pivot position
    assert sorted(order.tolist()) == list(range(m.n_species))
    A = P[np.ix_(order, order)].copy()
    for k in range(m.n_species):
        rows = np.nonzero(A[k + 1:, k])[0] + k + 1
        cols = np.nonzero(A[k, k + 1:])[0] + k + 1
        A[np.ix_(rows, cols)] = True
    assert np.array_equal(A, cp.fill) and cp.nnz_lu == int(A.sum())


@pytest.mark.parametrize("name", list(MECHS))
def test_programs_compute_f_and_solve_I_minus_cJ(oracle_lib, compiled, name):
    m, cp = compiled[name]
    lay, S, R = cp.lay, m.n_species, m.n_reactions
    om = oracle_lib.OracleMechanism(m)
    cells = synth.random_cells(S, 3, T_range=(210, 310), P_range=(1e3, 1e5), seed=31)
    rng = np.random.default_rng(32)
    for k in range(cells.n_cells):
        kt = oracle_lib.rate_constants(om, cells.T[k], cells.P[k])
        y = cells.y[:, k]
        Wd = np.full(lay["Wd_len"], np.nan)
        for i, v in cp.dconst:
            Wd[int(i)] = v
        Wd[lay["d_Y"]:lay["d_Y"] + S] = y
        Wd[lay["d_KT"]:lay["d_KT"] + R] = kt
        for j in range(R):                      # a2 rates, as the kernels form them before the program
            Wd[lay["d_RT"] + j] = kt[j] * np.prod(y[m.reac[j, :m.n_reac[j]]])
        pe.run(cp.progs["f"], Wd, cp.units["f"])
        J = oracle_lib.jacobian(om, kt, y)
        f = Wd[lay["d_F"]:lay["d_F"] + S]
        assert np.all(np.abs(f - oracle_lib.deriv(om, kt, y)) <= 1e-13 * (np.abs(J) @ np.abs(y) + 1e-300))
        for c in (1e-3, 7.5, 600.0):
            # the M program names the pair products by virtual slots above WL (on the
            # device they sit in Wd's rate and f slots, dead while M is formed)
            WL = np.full(max(lay["WL_len"], lay["L_P"] + len(cp.pair_rx)), np.nan)
            for i, v in cp.Lconst:
                WL[int(i)] = v
            WL[:lay["m_clear"]] = 0.0
            WL[cp.ludiag] = 1.0
            for pidx, j in enumerate(cp.pair_rx):   # -c k~_j times the pair's other reactants
                WL[lay["L_P"] + pidx] = -c * kt[j] * Wd[cp.pair_other[pidx, 0]] * Wd[cp.pair_other[pidx, 1]]
            pe.run(cp.progs["m"], WL, cp.units["m"])
            pe.run(cp.progs["lu"], WL, cp.units["lu"])
            Mk = np.eye(S) - c * J
            b = rng.standard_normal(S)
            for prog, Mref in ((("fwd", "bwd"), Mk), (("fwdT", "bwdT"), Mk.T)):
                W = WL.copy()
                W[lay["L_X"] + cp.pos] = b
                for p in prog:
                    pe.run(cp.progs[p], W, cp.units[p])
                x = -W[lay["L_X"] + cp.pos]             # the solves leave -x
                xr = np.linalg.solve(Mref, b)
                assert np.max(np.abs(x - xr)) <= 1e-10 * np.max(np.abs(xr)), (name, k, c, prog)


@pytest.mark.parametrize("name", list(MECHS))
def test_adjoint_programs_compute_J_transpose_mu(oracle_lib, compiled, name):
    m, cp = compiled[name]
    lay, adj, S = cp.lay, cp.adj, m.n_species
    om = oracle_lib.OracleMechanism(m)
    cells = synth.random_cells(S, 2, T_range=(210, 310), P_range=(1e3, 1e5), seed=33)
    for k in range(cells.n_cells):
        kt = oracle_lib.rate_constants(om, cells.T[k], cells.P[k])
        y = cells.y[:, k]
        # the cell's whole slice as the adjoint kernel sees it: the forward's Wd
        # (rounded to an even length) and WL, the adjoint's arrays, then the partials PP
        W = np.full(adj["a_PP"] + len(cp.pair_rx), np.nan)
        assert adj["a_MU"] == ((lay["Wd_len"] + 1) & ~1) + lay["WL_len"] and adj["a_PP"] == adj["Wda_len"]
        for i, v in np.concatenate([cp.dconst, cp.aconst]):
            W[int(i)] = v
        W[lay["d_Y"]:lay["d_Y"] + S] = y
        mu = np.random.default_rng(34 + k).standard_normal(S)
        W[adj["a_MU"]:adj["a_MU"] + S] = mu
        for pidx, j in enumerate(cp.pair_rx):
            W[adj["a_PP"] + pidx] = kt[j] * W[cp.pair_other[pidx, 0]] * W[cp.pair_other[pidx, 1]]
        pe.run(cp.progs["nudot"], W, cp.units["nudot"])
        pe.run(cp.progs["jt"], W, cp.units["jt"])
        J = oracle_lib.jacobian(om, kt, y)
        ref = J.T @ mu
        got = W[adj["a_JTM"]:adj["a_JTM"] + S]
        assert np.all(np.abs(got - ref) <= 1e-12 * (np.abs(J.T) @ np.abs(mu)))


def _half_warp_wavefronts(ops, n_units):
    """Shared-memory wavefronts of one pass's 8-byte operand accesses as the
    kernels' interpreter issues them: per operand (t, a, b, c), per half-warp,
    the most loaded bank pair (distinct slots with equal index mod 16), plus two
    for the op itself (a 32-lane 8-byte load)."""
    total = 0
    for p in range(ops.shape[0]):
        w = 2
        for r in range(4):
            for h in range(2):
                slots = set()
                for o in ops[p, 16 * h:16 * h + 16]:
                    t, a, b, c = (int(v) for v in o)
                    if t == pe.EMPTY:
                        continue          # empty slots touch one dummy or constant slot (a broadcast)
                    e = (t & ~pe.RECIP, a, None, None)[r] if t & pe.RECIP else (t, a, b, c)[r]
                    if e is not None:
                        slots.add(e)
                if slots:
                    w += int(np.bincount([e % 16 for e in slots], minlength=16).max())
        total += w
    return total / max(n_units, 1)


def _relabelled(ops, seed):
    """The same program with its slots renamed at random and each pass's ops
    dealt to lanes at random: what the passes cost without a bank layout."""
    rng = np.random.default_rng(seed)
    used = sorted({int(v) & ~pe.RECIP for o in ops.reshape(-1, 4) for v in o if int(v) != pe.EMPTY})
    perm = dict(zip(used, (int(x) for x in rng.permutation(used))))
    out = ops.copy()
    for idx in np.ndindex(ops.shape[:2]):
        t, a, b, c = (int(v) for v in ops[idx])
        if t != pe.EMPTY:
            out[idx] = (perm[t & ~pe.RECIP] | (t & pe.RECIP), perm[a], perm.get(b, b), perm.get(c, c))
    for p in range(out.shape[0]):
        out[p] = out[p][rng.permutation(out.shape[1])]
    return out


@pytest.mark.parametrize("name", ["tropo", "s128"])
@pytest.mark.parametrize("prog", ["lu", "fwd"])
def test_bank_layout_spreads_each_passs_operands(compiled, name, prog):
    # The compiler permutes the slots and deals each pass's ops to lanes so that
    # a pass's operand slots spread over the shared-memory bank pairs (an 8-byte
    # access is served per half-warp, one wavefront per distinct slot of the most
    # loaded bank pair).  For the 72/186 mechanism the LU passes cost about 16.7
    # wavefronts against about 24.4 for the same program with slots and lanes
    # dealt at random.
    m, cp = compiled[name]
    ops = cp.progs[prog]
    w = _half_warp_wavefronts(ops, ops.shape[0])
    w_random = np.mean([_half_warp_wavefronts(_relabelled(ops, s), ops.shape[0]) for s in range(2)])
    assert w <= 0.8 * w_random, (w, w_random)
