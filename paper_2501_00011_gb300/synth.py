"""Seeded synthetic inputs: mechanisms and cell states.

This module draws random tables and nothing else.  It holds none of the
solver's arithmetic (no rate constants, no derivatives, no integration), so
both the CUDA library and the CPU oracle can be fed from it without sharing
any of the method.

The workloads stand in for the condensed tropospheric mechanism (CB05) the
paper profiles in its Background section, which is not available here: a
gas-phase mass-action mechanism whose reactions take the general form
``c1*y1 + ... -> c_{m+1}*y_{m+1} + ...`` (Background, displayed reaction form)
with Arrhenius thermal rates and photolysis rates, over many independent grid
cells that each carry their own temperature, pressure and state
(Background, cells are independent; Implementations, Multi-cells).

Units: mixing ratios in mol/mol, T in K, P in Pa.  Thermal rate parameters
are for ``k = A * exp(-Ea/T) * (T/300)**B`` with ``Ea`` given as Ea/R in K;
for a reaction with n reactants ``A`` is in (cm^3 molec^-1)^(n-1) s^-1.
Photolysis reactions carry a first-order rate ``J`` in s^-1.

Stoichiometry (see the generator below): every species has an integer
"atom weight" w_i in {1..4} and every reaction conserves sum_i w_i * y_i, so
each synthetic mechanism has the linear invariant w^T nu = 0 that the tests
use as a pin.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# reaction kinds
THERMAL = 0      # Arrhenius rate, any number of reactants
PHOTOLYSIS = 1   # first-order, rate J (s^-1), optionally scaled per cell
TROE = 2         # pressure fall-off between a low- and a high-pressure Arrhenius limit
PRESSURE_SUM = 3   # an Arrhenius term plus a second one times the air number density
FALLOFF_SUM = 4    # an Arrhenius term plus a Lindemann fall-off term
# columns of Mechanism.ext: the second and third Arrhenius terms and the Troe broadening
EXT_A2, EXT_EA2, EXT_B2, EXT_A3, EXT_EA3, EXT_B3, EXT_FC, EXT_N = range(8)

MAX_REAC = 3
MAX_PROD = 8

SEED_MECHANISM = 20250011
SEED_CELLS = 20250012
SEED_PHOTOLYSIS = 20250013
SEED_LOSS_WEIGHTS = 20250014


@dataclass
class Mechanism:
    """Reaction tables of one mechanism (plain arrays, species indices 0-based)."""
    n_species: int
    kind: np.ndarray          # int32 [R]    THERMAL / PHOTOLYSIS
    n_reac: np.ndarray        # int32 [R]    1..MAX_REAC
    reac: np.ndarray          # int32 [R, MAX_REAC]  species index, -1 padding
    n_prod: np.ndarray        # int32 [R]    0..MAX_PROD
    prod: np.ndarray          # int32 [R, MAX_PROD]  species index, -1 padding
    yld: np.ndarray           # float64 [R, MAX_PROD] product yields, 0 padding
    A: np.ndarray             # float64 [R]
    Ea: np.ndarray            # float64 [R]  Ea/R in K
    B: np.ndarray             # float64 [R]
    J: np.ndarray             # float64 [R]  photolysis rate (0 for thermal)
    weights: np.ndarray | None = None   # int64 [S] conserved atom weights
    name: str = "mechanism"
    ext: np.ndarray | None = None       # float64 [R, 8] parameters of the pressure-dependent kinds (EXT_*)

    @property
    def n_reactions(self) -> int:
        return int(self.kind.shape[0])

    @property
    def photolysis_index(self) -> np.ndarray:
        """Reaction indices of the photolysis reactions, in reaction order."""
        return np.nonzero(self.kind == PHOTOLYSIS)[0].astype(np.int32)


@dataclass
class Cells:
    """State of a batch of cells; y is [n_species, n_cells], cell index unit stride."""
    T: np.ndarray             # float64 [C]
    P: np.ndarray             # float64 [C]
    y: np.ndarray             # float64 [S, C]
    # per-cell photolysis rates [n_phot, C] (None: every cell uses the mechanism's J)
    J: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.T.shape[0])


def empty_mechanism(n_species: int, n_reactions: int, name: str = "mechanism") -> Mechanism:
    R = n_reactions
    return Mechanism(
        n_species=n_species,
        kind=np.zeros(R, np.int32),
        n_reac=np.zeros(R, np.int32),
        reac=np.full((R, MAX_REAC), -1, np.int32),
        n_prod=np.zeros(R, np.int32),
        prod=np.full((R, MAX_PROD), -1, np.int32),
        yld=np.zeros((R, MAX_PROD), np.float64),
        A=np.zeros(R), Ea=np.zeros(R), B=np.zeros(R), J=np.zeros(R),
        name=name, ext=np.zeros((R, 8)),
    )


def rate_ext(m: Mechanism) -> np.ndarray:
    """m.ext, or zeros for a mechanism without pressure-dependent kinds."""
    return np.zeros((m.n_reactions, 8)) if m.ext is None else np.asarray(m.ext, np.float64)


def mechanism_from_list(n_species: int, reactions: list[dict], name: str = "mechanism") -> Mechanism:
    """Build a mechanism from a list of dicts.

    Each dict: ``reac`` (list of species, repeats allowed), ``prod`` (list of
    species), optional ``yld`` (list of yields, default 1.0 each) and either
    ``J`` (photolysis) or ``A`` [, ``Ea``, ``B``] (thermal), the latter with an
    optional ``kind`` (TROE, PRESSURE_SUM, FALLOFF_SUM) and its parameters
    ``A2``, ``Ea2``, ``B2``, ``A3``, ``Ea3``, ``B3``, ``Fc``, ``N`` (default 0;
    Fc 0.6 and N 1 for TROE).
    """
    m = empty_mechanism(n_species, len(reactions), name)
    for j, rx in enumerate(reactions):
        reac = list(rx["reac"])
        prod = list(rx.get("prod", []))
        yld = list(rx.get("yld", [1.0] * len(prod)))
        assert 1 <= len(reac) <= MAX_REAC and len(prod) <= MAX_PROD and len(yld) == len(prod)
        m.n_reac[j] = len(reac)
        m.reac[j, :len(reac)] = reac
        m.n_prod[j] = len(prod)
        m.prod[j, :len(prod)] = prod
        m.yld[j, :len(prod)] = yld
        if "J" in rx:
            m.kind[j] = PHOTOLYSIS
            m.J[j] = rx["J"]
        else:
            m.kind[j] = rx.get("kind", THERMAL)
            m.A[j] = rx["A"]
            m.Ea[j] = rx.get("Ea", 0.0)
            m.B[j] = rx.get("B", 0.0)
            troe = m.kind[j] == TROE
            m.ext[j] = [rx.get("A2", 0.0), rx.get("Ea2", 0.0), rx.get("B2", 0.0), rx.get("A3", 0.0),
                        rx.get("Ea3", 0.0), rx.get("B3", 0.0), rx.get("Fc", 0.6 if troe else 0.0),
                        rx.get("N", 1.0 if troe else 0.0)]
    return m


# ---------------------------------------------------------------------------
# random condensed-tropospheric-style mechanisms
# ---------------------------------------------------------------------------

def _partitions(total: int, max_parts: int = 3, max_part: int = 4) -> list[tuple[int, ...]]:
    """All multisets of 1..max_parts integers in [1, max_part] summing to total."""
    out = []

    def rec(rem, parts, lo):
        if rem == 0 and parts:
            out.append(tuple(parts))
            return
        if len(parts) == max_parts:
            return
        for p in range(lo, min(rem, max_part) + 1):
            rec(rem - p, parts + [p], p)

    rec(total, [], 1)
    return out


def random_mechanism(n_species: int, n_reactions: int, n_unimolecular: int, n_photolysis: int,
                     seed: int = SEED_MECHANISM, n_hubs: int | None = None,
                     name: str | None = None) -> Mechanism:
    """Seeded synthetic gas-phase mechanism.

    Recipe (stated so the workload can be re-created without this code):

    * Species get conserved integer weights w in {1,2,3,4} with probabilities
      0.4/0.3/0.2/0.1 (at least two species of each weight).
    * A few "hub" species (default max(4, S//10)) play the role of the radical
      oxidants and NOx of a tropospheric mechanism: the second reactant of a
      bimolecular reaction is a hub with probability 0.7, and a product is drawn
      among hubs with probability 0.3.  Species indices are shuffled so hubs are
      not contiguous.
    * ``n_unimolecular`` reactions have one reactant; the first ``n_photolysis``
      of them are photolysis (J log-uniform in [1e-5, 1e-2] s^-1), the rest are
      thermal.  The remaining reactions are bimolecular; one in ten is the
      self-reaction 2A.
    * Products: 1-3 distinct species, none of them a reactant, unit yields,
      chosen so that the summed product weight equals the summed reactant weight.
    * Every species takes part in at least one reaction.
    * Thermal parameters: log10 A ~ U[-14,-10], Ea/R ~ U[0,2000] K, B ~ U[-2,2].
    * Reaction order is shuffled.
    """
    S, R = n_species, n_reactions
    assert 0 <= n_photolysis <= n_unimolecular <= R
    rng = np.random.Generator(np.random.PCG64([seed, S, R]))
    if n_hubs is None:
        n_hubs = max(4, S // 10)

    w = rng.choice([1, 2, 3, 4], size=S, p=[0.4, 0.3, 0.2, 0.1])
    for v in (1, 2, 3, 4):          # at least two species of each weight
        while np.count_nonzero(w == v) < 2:
            cand = np.nonzero(np.bincount(w, minlength=5)[w] > 2)[0]
            w[rng.choice(cand)] = v
    perm = rng.permutation(S)
    hubs = perm[:n_hubs]
    is_hub = np.zeros(S, bool)
    is_hub[hubs] = True
    nonhub = np.nonzero(~is_hub)[0]
    by_weight = {v: np.nonzero(w == v)[0] for v in (1, 2, 3, 4)}
    hub_by_weight = {v: np.intersect1d(by_weight[v], hubs) for v in (1, 2, 3, 4)}

    def pick_products(reactants):
        total = int(sum(w[r] for r in reactants))
        parts_opts = [p for p in _partitions(total) if len(p) <= 3]
        for _ in range(200):
            parts = parts_opts[rng.integers(len(parts_opts))]
            chosen = []
            ok = True
            for v in parts:
                pool = by_weight[v]
                if rng.random() < 0.3 and hub_by_weight[v].size:
                    pool = hub_by_weight[v]
                pool = np.setdiff1d(pool, list(reactants) + chosen)
                if pool.size == 0:
                    ok = False
                    break
                chosen.append(int(rng.choice(pool)))
            if ok:
                return chosen
        raise RuntimeError("could not balance a reaction")

    m = empty_mechanism(S, R, name or f"synthetic_{S}sp_{R}rx")
    for j in range(R):
        if j < n_unimolecular:
            reactants = [int(rng.choice(nonhub if rng.random() < 0.8 else hubs))]
        else:
            a = int(rng.choice(nonhub if rng.random() < 0.75 else hubs))
            if rng.random() < 0.1:
                reactants = [a, a]
            else:
                pool = hubs if rng.random() < 0.7 else np.arange(S)
                pool = pool[pool != a]
                reactants = [a, int(rng.choice(pool))]
        products = pick_products(reactants)
        m.n_reac[j] = len(reactants)
        m.reac[j, :len(reactants)] = reactants
        m.n_prod[j] = len(products)
        m.prod[j, :len(products)] = products
        m.yld[j, :len(products)] = 1.0
        if j < n_photolysis:
            m.kind[j] = PHOTOLYSIS
            m.J[j] = 10.0 ** rng.uniform(-5.0, -2.0)
        else:
            m.kind[j] = THERMAL
            m.A[j] = 10.0 ** rng.uniform(-14.0, -10.0)
            m.Ea[j] = rng.uniform(0.0, 2000.0)
            m.B[j] = rng.uniform(-2.0, 2.0)

    # every species takes part: swap an uncovered species into a product slot of
    # equal weight whose current occupant appears elsewhere too
    for _ in range(10 * S):
        count = np.zeros(S, int)
        for j in range(R):
            for s in m.reac[j, :m.n_reac[j]]:
                count[s] += 1
            for s in m.prod[j, :m.n_prod[j]]:
                count[s] += 1
        missing = np.nonzero(count == 0)[0]
        if missing.size == 0:
            break
        s = int(missing[0])
        done = False
        for j in rng.permutation(R):
            reac = set(m.reac[j, :m.n_reac[j]].tolist())
            prods = m.prod[j, :m.n_prod[j]].tolist()
            if s in reac:
                continue
            for k, p in enumerate(prods):
                if w[p] == w[s] and count[p] > 1 and s not in prods:
                    m.prod[j, k] = s
                    done = True
                    break
            if done:
                break
        if not done:
            raise RuntimeError("could not cover every species")
    else:
        raise RuntimeError("species coverage did not converge")

    order = rng.permutation(R)
    for name_ in ("kind", "n_reac", "reac", "n_prod", "prod", "yld", "A", "Ea", "B", "J"):
        setattr(m, name_, np.ascontiguousarray(getattr(m, name_)[order]))
    m.weights = w.astype(np.int64)
    return m


def random_cells(n_species: int, n_cells: int, T_range=(250.0, 300.0), P_range=(1e5, 1e5),
                 y_range=(1e-12, 1e-6), seed: int = SEED_CELLS) -> Cells:
    """Seeded cell batch: T uniform, P log-uniform, y log-uniform per species and cell."""
    rng = np.random.Generator(np.random.PCG64([seed, n_species, n_cells]))
    T = rng.uniform(T_range[0], T_range[1], size=n_cells)
    if P_range[0] == P_range[1]:
        P = np.full(n_cells, float(P_range[0]))
    else:
        P = 10.0 ** rng.uniform(np.log10(P_range[0]), np.log10(P_range[1]), size=n_cells)
    y = 10.0 ** rng.uniform(np.log10(y_range[0]), np.log10(y_range[1]), size=(n_species, n_cells))
    return Cells(T=T, P=P, y=np.ascontiguousarray(y))


def photolysis_scale(n_cells: int, night_fraction: float = 0.3, seed: int = SEED_PHOTOLYSIS) -> np.ndarray:
    """Per-cell photolysis scale s_c: 0 for a seeded night fraction, else U(0, 1]."""
    rng = np.random.Generator(np.random.PCG64([seed, n_cells]))
    s = 1.0 - rng.uniform(0.0, 1.0, size=n_cells)          # (0, 1]
    night = rng.random(n_cells) < night_fraction
    s[night] = 0.0
    return s


def loss_weights(n_species: int, n_cells: int, seed: int = SEED_LOSS_WEIGHTS) -> np.ndarray:
    """Weights of the scalar loss on final concentrations, U[0,1], shape [S, C]."""
    rng = np.random.Generator(np.random.PCG64([seed, n_species, n_cells]))
    return rng.uniform(0.0, 1.0, size=(n_species, n_cells))


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mech: Mechanism
    cells: Cells
    dt: float
    n_steps: int
    rtol: float
    atol: float
    lu_precision: int = 64


def mechanism_small() -> Mechanism:
    """20 species / 40 reactions: 12 unimolecular of which 4 photolysis, 28 bimolecular."""
    return random_mechanism(20, 40, 12, 4, name="synthetic_20sp_40rx")


def mechanism_tropo() -> Mechanism:
    """72 species / 186 reactions: 56 unimolecular (30%) of which 19 photolysis, 130 bimolecular."""
    return random_mechanism(72, 186, 56, 19, name="synthetic_72sp_186rx")


def mechanism_tropo_pressure() -> Mechanism:
    """The 72/186 mechanism with 18 of its bimolecular thermal reactions made
    pressure-dependent, about as many as a condensed tropospheric mechanism
    has: 12 Troe fall-off reactions (log10 k0 ~ U[-32,-29] cm^6 s^-1,
    k0 temperature exponent B ~ U[-4,-1], log10 kinf ~ U[-12,-10], kinf exponent
    ~ U[-1,0], no activation energies, Fc = 0.6, N = 1), three k_a + k_b [M]
    (log10 A ~ U[-13.5,-12.5], Ea/R ~ U[-600,0] K; log10 A2 ~ U[-33.5,-32.5],
    Ea2/R ~ U[-1000,0] K) and three k_a + k_c [M] / (1 + k_c [M] / k_b)
    (log10 A ~ U[-14.5,-13.5], Ea/R ~ U[-600,0]; log10 A2 ~ U[-17.5,-16.5],
    Ea2/R ~ U[-2400,-2000]; log10 A3 ~ U[-34,-33], Ea3/R ~ U[-1500,-1200]).
    Species, stoichiometry and sparsity are those of mechanism_tropo()."""
    m = mechanism_tropo()
    m.name = "synthetic_72sp_186rx_pressure"
    rng = np.random.Generator(np.random.PCG64([SEED_MECHANISM, 72, 186, 2]))
    cand = np.nonzero((m.kind == THERMAL) & (m.n_reac == 2))[0]
    pick = rng.choice(cand, 18, replace=False)
    ext = np.zeros((m.n_reactions, 8))
    for i, j in enumerate(pick):
        if i < 12:
            m.kind[j] = TROE
            m.A[j], m.Ea[j], m.B[j] = 10.0 ** rng.uniform(-32.0, -29.0), 0.0, rng.uniform(-4.0, -1.0)
            ext[j, EXT_A2], ext[j, EXT_EA2], ext[j, EXT_B2] = 10.0 ** rng.uniform(-12.0, -10.0), 0.0, rng.uniform(-1.0, 0.0)
            ext[j, EXT_FC], ext[j, EXT_N] = 0.6, 1.0
        elif i < 15:
            m.kind[j] = PRESSURE_SUM
            m.A[j], m.Ea[j], m.B[j] = 10.0 ** rng.uniform(-13.5, -12.5), rng.uniform(-600.0, 0.0), 0.0
            ext[j, EXT_A2], ext[j, EXT_EA2] = 10.0 ** rng.uniform(-33.5, -32.5), rng.uniform(-1000.0, 0.0)
        else:
            m.kind[j] = FALLOFF_SUM
            m.A[j], m.Ea[j], m.B[j] = 10.0 ** rng.uniform(-14.5, -13.5), rng.uniform(-600.0, 0.0), 0.0
            ext[j, EXT_A2], ext[j, EXT_EA2] = 10.0 ** rng.uniform(-17.5, -16.5), rng.uniform(-2400.0, -2000.0)
            ext[j, EXT_A3], ext[j, EXT_EA3] = 10.0 ** rng.uniform(-34.0, -33.0), rng.uniform(-1500.0, -1200.0)
    m.ext = ext
    return m


def workload_pressure(n_cells: int = 10_000) -> Workload:
    """One 600 s step of the pressure-dependent 72/186 mechanism over cells
    spanning the troposphere and lower stratosphere: T in [200, 310] K, P in
    [1e3, 1.05e5] Pa (log-uniform), so the fall-off reactions run from near
    their low-pressure to near their high-pressure limits."""
    m = mechanism_tropo_pressure()
    c = random_cells(m.n_species, n_cells, T_range=(200.0, 310.0), P_range=(1e3, 1.05e5))
    return Workload("tropo_pressure_72sp_186rx", m, c, 600.0, 1, 1e-4, 1e-10)


def workload_small(n_cells: int = 10) -> Workload:
    """One 600 s step of the 20/40 mechanism over 10 cells, rtol 1e-8, atol 1e-14."""
    m = mechanism_small()
    c = random_cells(m.n_species, n_cells, T_range=(250.0, 300.0), P_range=(1e5, 1e5))
    return Workload("small_20sp_40rx", m, c, 600.0, 1, 1e-8, 1e-14)


def workload_tropo(n_cells: int = 10_000) -> Workload:
    """One 600 s step of the 72/186 mechanism over 10,000 cells, rtol 1e-4, atol 1e-10."""
    m = mechanism_tropo()
    c = random_cells(m.n_species, n_cells, T_range=(220.0, 310.0), P_range=(2e4, 1e5))
    return Workload("tropo_72sp_186rx", m, c, 600.0, 1, 1e-4, 1e-10)


def workload_batching(n_cells: int = 50_000) -> Workload:
    """Six 600 s steps, 50,000 cells, T in [200,320] K, per-cell photolysis 0 (night)..J."""
    m = mechanism_tropo()
    c = random_cells(m.n_species, n_cells, T_range=(200.0, 320.0), P_range=(2e4, 1e5))
    s = photolysis_scale(n_cells)
    c.J = np.ascontiguousarray(m.J[m.photolysis_index][:, None] * s[None, :])
    c.meta["photolysis_scale"] = s
    return Workload("tropo_batching_50k", m, c, 600.0, 6, 1e-4, 1e-10)


def workload_precision(n_cells: int = 50_000) -> Workload:
    """The batching cells for one 600 s step with the LU factor/solve in FP32."""
    w = workload_batching(n_cells)
    w.name, w.n_steps, w.lu_precision = "tropo_fp32lu_50k", 1, 32
    return w


def workload_adjoint(n_cells: int = 2_048) -> Workload:
    """Four 600 s steps over 2,048 cells for the discrete adjoint."""
    m = mechanism_tropo()
    c = random_cells(m.n_species, n_cells, T_range=(220.0, 310.0), P_range=(2e4, 1e5))
    return Workload("tropo_adjoint_2k", m, c, 600.0, 4, 1e-4, 1e-10)


def subset(cells: Cells, idx) -> Cells:
    """A cell subset (copies), e.g. a bounded sample for a CPU timing."""
    idx = np.asarray(idx)
    return Cells(T=cells.T[idx].copy(), P=cells.P[idx].copy(),
                 y=np.ascontiguousarray(cells.y[:, idx]),
                 J=None if cells.J is None else np.ascontiguousarray(cells.J[:, idx]),
                 meta=dict(cells.meta))
