"""CPU replay of the compiled warp programs (test helper).

The library's host-side mechanism compiler turns a reaction table into
32-lane "pass" programs that the kernels interpret: each op of a pass is
t <- a * b + c on per-cell slots (or t <- -1 / a for a reciprocal op), all ops
of a pass reading before any writes.  tests/native/progdump.cpp runs that
compiler on the CPU and writes the programs out; this module builds it,
parses its output and replays the programs in numpy, checking on the way
that no pass has a read/write or write/write conflict and that every slot
index lies inside the cell's arrays.
"""
import ctypes
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_00011_gb300", "csrc")
EMPTY, RECIP = 0xFFFF, 0x8000
PROGRAMS = ("f", "m", "lu", "fwd", "bwd", "nudot", "jt", "fwdT", "bwdT")
LAYOUT = "Wd_len d_Y d_KT d_RT d_F d_ONE d_ZERO WL_len L_LU L_X L_P L_ZERO nnz_lu m_clear".split()
ADJ = "Wda_len a_MU a_NM a_PP a_JTM a_G".split()


def build_dumper(outdir):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(outdir, "progdump")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "native", "progdump.cpp"),
                    os.path.join(CSRC, "mechanism.cpp"), "-L", os.path.join(cuda, "lib64"), "-lcudart", "-o", exe],
                   check=True)
    return exe


class Compiled:
    """Layout, tables and programs of one compiled mechanism."""

    def __init__(self, exe, mech, workdir):
        from paper_2501_00011_gb300 import chemgpu
        rx = chemgpu.reactions_from_synth(mech)
        src, out = os.path.join(workdir, f"{mech.name}.bin"), os.path.join(workdir, f"{mech.name}.txt")
        with open(src, "wb") as fh:
            fh.write(np.array([mech.n_species, mech.n_reactions], np.int32).tobytes())
            fh.write(bytes(memoryview(rx))[:ctypes.sizeof(chemgpu.Reaction) * mech.n_reactions])
        r = subprocess.run([exe, src, out], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"progdump failed: {r.stdout}{r.stderr}")
        lines = open(out).read().split("\n")
        D, self.progs, i = {}, {}, 0
        while i < len(lines):
            L = lines[i].split()
            if not L:
                i += 1
                continue
            if L[0] in PROGRAMS:
                n = int(L[1])
                body = [list(map(int, lines[i + 1 + k].split())) for k in range(32 * n)]
                self.progs[L[0]] = np.array(body, np.int64).reshape(n, 32, 4) if n else np.zeros((0, 32, 4), np.int64)
                i += 1 + 32 * n
                continue
            D[L[0]] = L[1:]
            i += 1
        self.lay = dict(zip(LAYOUT, map(int, D["layout"])))
        self.adj = dict(zip(ADJ, map(int, D["adj"])))
        S = mech.n_species
        self.pos = np.array(D["pos"], int)
        self.ludiag = np.array(D["ludiag"], int)
        self.pair_rx = np.array(D.get("pairrx", []), int)
        self.pair_other = np.array(D.get("pairother", []), int).reshape(-1, 2)
        self.dconst = np.array(D.get("dconst", []), float).reshape(-1, 2)
        self.Lconst = np.array(D.get("Lconst", []), float).reshape(-1, 2)
        self.aconst = np.array(D.get("aconst", []), float).reshape(-1, 2)
        self.fill = np.array(D["fill"], int).reshape(S, S).astype(bool)
        self.nnz_jac, self.nnz_lu = map(int, D["info"])
        # per pass: 0 single FMA pass, 1 / 2 first / second pass of an independent pair, 3 reciprocals
        self.units = {k: np.array(D.get("units_" + k, []), int) for k in PROGRAMS}


def run(ops, W, units=None):
    """Replay one program on the slot array W in place (race and bounds checked).

    units (the compiler's per-pass unit kinds): the two passes of a pair run
    as one group of 64 ops, which the kernels execute with every load before
    the stores, so the check covers both passes together."""
    n = W.shape[0]
    groups, p = [], 0
    while p < ops.shape[0]:
        if units is not None and len(units) and units[p] == 1:
            assert units[p + 1] == 2, ("unpaired pair unit", p)
            groups.append(np.concatenate([ops[p], ops[p + 1]]))
            p += 2
        else:
            assert units is None or not len(units) or units[p] in (0, 3), ("stray pair unit", p)
            groups.append(ops[p])
            p += 1
    for p, group in enumerate(groups):
        writes, reads, new = set(), set(), {}
        for t, a, b, c in group:
            t, a, b, c = int(t), int(a), int(b), int(c)
            if t == EMPTY:
                continue
            if t & RECIP:
                t &= ~RECIP
                srcs = (a,)
            else:
                srcs = (a, b, c)
            assert max((t,) + srcs) < n, ("slot out of range", p, t, srcs, n)
            assert t not in writes and t not in reads, ("write conflict in a pass", p, t)
            assert not any(x in writes for x in srcs), ("read after write in a pass", p, srcs)
            writes.add(t)
            reads.update(srcs)
            new[t] = -1.0 / W[a] if len(srcs) == 1 else W[a] * W[b] + W[c]
        for t, v in new.items():
            W[t] = v
