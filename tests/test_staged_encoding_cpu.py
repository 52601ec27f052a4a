"""The register-tile plan's encoding, checked without a GPU: the records that
sim_plan_staged_ops returns (the ones the staged kernel executes) are run by
a plain Python model of what each record means, and the result must equal
the FP64 oracle's state for the original circuit.

The model restates the op semantics from the header's description, not the
kernel's code: a tile is the 2^M amplitudes sharing every qubit outside the
pass's local set; thread i and register k of layout l address local index
sum of bit(i, b) 2^thr(l, b) + sum of bit(k, j) 2^reg(l, j); an exchange
record updates the amplitude pairs (k, k | 2^arg) of every thread whose
conditions hold; a diagonal record multiplies the amplitudes whose
conditions (and target bit) hold; a ramp multiplies the amplitudes whose
shared qubit is 1 by the product of the thread's and the register's table
entries.  Layout tables: layout 0 keeps local bit 0 (complex64) and the top
register bits in registers; layout l >= 1 takes a window of register bits
starting at 1 (complex64) or 0, RB (M - 8) bits per layout, clamped to the
top; thread bits are the remaining local bits in ascending order.

This catches planner mistakes (a wrong mask, a layout that does not hold
the target, a ramp that joins phases it must not, padding that breaks a
record) on the CPU; the GPU tests check the kernel against the oracle."""
import math

import numpy as np
import pytest

from paper_1805_00988_gb300 import circuits as C

THR_BITS = 8


def reg_local(M, RB, VEC, l, j):
    if l == 0:
        return (0 if j == 0 else M - RB + j) if VEC == 2 else (M - RB + j)
    s = (1 if VEC == 2 else 0) + RB * (l - 1)
    return min(s, M - RB) + j


def thr_local(M, RB, VEC, l, i):
    regs = {reg_local(M, RB, VEC, l, j) for j in range(RB)}
    free = [b for b in range(M) if b not in regs]
    return free[i]


def layout_index(M, RB, VEC, l):
    """local index of (thread, register): shape (256, 2^RB)"""
    tid = np.arange(1 << THR_BITS)[:, None]
    k = np.arange(1 << RB)[None, :]
    idx = np.zeros((1 << THR_BITS, 1 << RB), dtype=np.int64)
    for i in range(THR_BITS):
        idx += ((tid >> i) & 1) << thr_local(M, RB, VEC, l, i)
    for j in range(RB):
        idx += ((k >> j) & 1) << reg_local(M, RB, VEC, l, j)
    return idx


def bits_of(mask, count):
    return np.array([(int(mask) >> k) & 1 for k in range(count)], dtype=bool)


def run_encoded(psi, n, ops, info):
    psi = psi.copy()
    tid = np.arange(1 << THR_BITS)
    for row in info:
        first, count, M, RB, VEC, nh = (int(v) for v in row[:6])
        local = list(range(5)) + [int(q) for q in row[6:6 + nh]]
        outer = [q for q in range(n) if q not in local]
        RA = 1 << RB
        nrec = (RA + 32 + 3) // 4
        tables = {}
        lidx = np.arange(1 << M)
        gl = np.zeros(1 << M, dtype=np.int64)
        for b, q in enumerate(local):
            gl |= ((lidx >> b) & 1) << q
        for t in range(1 << (n - M)):
            base = 0
            for i, q in enumerate(outer):
                base |= ((t >> i) & 1) << q
            loc = psi[base | gl].copy()
            layout = 0
            p = 0
            while p < count:
                o = ops[first + p]
                kind = int(o["kind"])
                if kind == 0:
                    layout = int(o["arg"])
                    p += 1
                    continue
                if kind == 8:
                    p += 1
                    continue
                if layout not in tables:
                    tables[layout] = layout_index(M, RB, VEC, layout)
                idx = tables[layout]
                if kind == 7:
                    ent = np.array([complex(ops[first + p + (e >> 2)]["m"][2 * (e & 3)],
                                            ops[first + p + (e >> 2)]["m"][2 * (e & 3) + 1]) for e in range(4 * nrec)])
                    qt = ((tid & int(o["thr_t"])) != 0) | ((base & int(o["out_t"])) != 0)
                    one = np.where(qt[:, None], True, bits_of(o["km_t"], RA)[None, :])
                    F = ent[RA + (tid & 15)] * ent[RA + 16 + ((tid >> 4) & 15)]
                    G = F[:, None] * ent[:RA][None, :]
                    loc[idx[one]] *= G[one]
                    p += nrec
                    continue
                m = o["m"]
                A, B, Cc, D = (complex(m[2 * i], m[2 * i + 1]) for i in range(4))
                tok = ((tid & int(o["thr_c"])) == int(o["thr_c"])) & ((base & int(o["out_c"])) == int(o["out_c"]))
                kmc = bits_of(o["km_c"], RA)
                if kind in (1, 2, 3):
                    J = int(o["arg"])
                    act = np.ones((len(tid), RA), dtype=bool) if int(o["plain"]) else (tok[:, None] & kmc[None, :])
                    for k in range(RA):
                        if (k >> J) & 1:
                            continue
                        sel = act[:, k]
                        il, ih = idx[sel, k], idx[sel, k | (1 << J)]
                        lo, hi = loc[il].copy(), loc[ih].copy()
                        if kind == 1:
                            loc[il], loc[ih] = A * lo + B * hi, Cc * lo + D * hi
                        elif kind == 2:
                            loc[il], loc[ih] = B * hi, Cc * lo
                        else:
                            loc[il], loc[ih] = hi, lo
                else:
                    ctb = ((tid & int(o["thr_t"])) != 0) | ((base & int(o["out_t"])) != 0)
                    cond = tok[:, None] & kmc[None, :]
                    one = np.where(ctb[:, None], cond, cond & bits_of(o["km_t"], RA)[None, :])
                    if kind == 6:
                        loc[idx[one]] *= -1.0
                    elif kind == 5:
                        loc[idx[one]] *= D
                    else:
                        loc[idx[cond]] *= np.where(one[cond], D, A)
                p += 1
            assert layout == 0, "a pass must end in the I/O layout"
            psi[base | gl] = loc
    return psi


def phase_runs(n, seed):
    rng = np.random.default_rng(seed)
    parts = [C.gate("h", q) for q in range(n)]
    for _ in range(8):
        q = int(rng.integers(0, n))
        partners = [int(m) for m in rng.choice([m for m in range(n) if m != q], size=int(rng.integers(3, n)),
                                               replace=False)]
        partners += partners[:2]
        for m in partners:
            parts.append(C.gate("p", q, controls=(m,), params=(float(rng.uniform(-math.pi, math.pi)),)))
        for t in rng.choice(n, size=3, replace=False):
            parts.append(C.gate("u3", int(t), params=tuple(float(x) for x in rng.uniform(0, 2 * math.pi, 3))))
    return C.concat(parts)


@pytest.mark.parametrize("dtype,n,tile", [(0, 12, 11), (0, 13, 13), (0, 14, 12), (0, 15, 13), (1, 12, 11),
                                          (1, 14, 12), (1, 13, 11)])
def test_encoded_plan_matches_oracle(orc, dtype, n, tile):
    from paper_1805_00988_gb300 import sim
    rng_gates = C.random_gates(n, 250, seed=n * 5 + tile + dtype, max_ctrl=2)
    sw = rng_gates["name"] == "swap"
    rng_gates["nctrl"][sw] = np.minimum(rng_gates["nctrl"][sw], 1)
    gates = C.concat([rng_gates, C.qft_paper(n), phase_runs(n, seed=n + tile), C.haar_cz(n, 2, seed=tile)])
    ops, info = sim.sim_plan_staged_ops(n, dtype, sim.to_sim_gates(gates), tile)
    assert (ops["kind"] == 7).any(), "the circuit should produce phase ramps"
    psi = C.random_state(n, seed=n + 2 * tile)
    got = run_encoded(psi, n, ops, info)
    ref = orc.apply_circuit(psi, gates)
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_ramp_records_stay_inside_one_staged_chunk():
    """The kernel stages records in chunks of 64 per pass; a ramp's records
    must not cross a chunk boundary (the planner pads with no-op records)."""
    from paper_1805_00988_gb300 import sim
    g = C.concat([C.qft_paper(16), phase_runs(16, seed=3), C.qft_paper(16)])
    for dtype, tile in ((0, 13), (0, 11), (1, 12)):
        ops, info = sim.sim_plan_staged_ops(16, dtype, sim.to_sim_gates(g), tile)
        for row in info:
            first, count, M, RB = (int(v) for v in row[:4])
            nrec = ((1 << RB) + 32 + 3) // 4
            kinds = ops["kind"][first:first + count]
            for p in np.nonzero(kinds == 7)[0]:
                assert p // 64 == (p + nrec - 1) // 64
                assert np.all(kinds[p + 1:p + nrec] == 8)
