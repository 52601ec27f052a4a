"""Small single-kernel workloads for profiler captures.

    python -m paper_1805_00988_gb300.kernel_cases k6        # fused 6-qubit blocks, 27 qubits
    python -m paper_1805_00988_gb300.kernel_cases pergate   # CNOT / CZ / SWAP, low qubit 3, 8, 17, 25; 27 qubits
    python -m paper_1805_00988_gb300.kernel_cases batch     # 512 variational circuits, one persistent launch
    python -m paper_1805_00988_gb300.kernel_cases c128      # complex128 fused 4-qubit blocks, 27 qubits (2 GiB)
    python -m paper_1805_00988_gb300.kernel_cases channel   # density-matrix channel passes, 13-qubit rho (26-qubit register)
    python -m paper_1805_00988_gb300.kernel_cases qft       # App. A QFT in register tiles (phase ramps), 26 qubits

Each case holds a few GB on the device at most (a 27-qubit complex64 state
is 1 GiB, 8x the L2), so a full ncu capture of one launch ends in a minute
or two.  The work goes through the C ABI like every other caller's.
"""
from __future__ import annotations

import sys


def main(argv=None):
    import torch

    from . import circuits as C
    from . import sim

    mode = (argv or sys.argv[1:] or ["k6"])[0]
    if mode == "k6":
        st = sim.State(27, "c64")
        st.apply(C.haar_cz(27, 3, seed=1234), plan="fused", fuse_k=6)
    elif mode == "pergate":
        st = sim.State(27, "c64")
        st.apply(C.concat([C.gate("h", q) for q in range(27)]), plan="staged")
        for c in (3, 8, 17, 25):
            t = 12 if c == 17 else 17
            st.apply(C.concat([C.gate("x", t, controls=(c,)), C.gate("z", t, controls=(c,)),
                               C.gate("swap", t, target2=c)]), plan="per_gate")
    elif mode == "c128":
        st = sim.State(27, "c128")
        st.apply(C.haar_cz(27, 3, seed=1234), plan="fused", fuse_k=4)
    elif mode == "qft":
        st = sim.State(26, "c64")
        st.apply(C.qft_paper(26), plan="staged")
    elif mode == "channel":
        rho = sim.DensityMatrix(13, "c64")
        rho.apply(C.haar_cz(13, 1, seed=1234), plan="per_gate")
        for t in (0, 5, 12):
            rho.apply_channel("depolarizing", 0.01, t)
            rho.apply_channel("amplitude_damping", 0.02, t)
        rho.close()
    elif mode == "batch":
        ns, offs, bg = C.variational(512, 8, 20, 4, 12, seed=1234)
        b = sim.Batch(ns, offs, bg)
        b.run()
        b.run()
        b.close()
    else:
        raise SystemExit("unknown case %r (k6, pergate, batch, c128, channel, qft)" % mode)
    torch.cuda.synchronize()
    print("ok", mode)


if __name__ == "__main__":
    main()
