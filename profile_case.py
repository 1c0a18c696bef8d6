"""Small, self-contained cases for ncu captures (a harness beside bench.py).

    python profile_case.py --rows 32            # TFIM-20 x10 energy+gradient
    python profile_case.py --workload noisy16   # 16-qubit noisy trajectories
    python profile_case.py --workload hea10     # 10-qubit complex128 ansatz
    python profile_case.py --workload qgt --qubits 16 --rows 1
                                                          # geometric tensor of the TFIM ansatz (10 layers)
    python profile_case.py --workload tn40 --rows 64 --precision 1
                                                          # whole 40-qubit testbed network, tensor-core steps
    python profile_case.py --workload qaoa --qubits 26 --rows 1 --layers 3
                                                          # MaxCut QAOA on a random 3-regular graph
    python profile_case.py --workload cone200 --rows 1 --cluster 8
                                                          # <Z99 Z100> light cone of the 200-qubit brickwork
    python profile_case.py --workload hea10_one --steps 4
                                                          # the 10-qubit ansatz, state and observables in one launch
"""
import numpy as np
import argparse

import torch

from paper_2205_10091_b300 import native as nt
from paper_2205_10091_b300 import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tfim20", choices=["tfim20", "noisy16", "hea10", "hea10_one", "qgt", "tn40", "qaoa", "cone200"])
    ap.add_argument("--rows", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--qubits", type=int, default=16)
    ap.add_argument("--precision", type=int, default=1, help="tn40: 0 FP32, 1 TF32X3, 2 BF16X6")
    ap.add_argument("--layers", type=int, default=3, help="qaoa: layers p")
    ap.add_argument("--cluster", type=int, default=8, help="cone200: CTAs per instance of the fused launch (1 = off)")
    ap.add_argument("--specialize", action="store_true", help="tfim20, qaoa, noisy16: pass kernels compiled for the circuit")
    args = ap.parse_args()
    if args.workload == "tfim20":
        circ, theta, ham = W.tfim_workload(20, 10, args.rows)
        c = nt.Circuit(circ, specialize=args.specialize)
        H = nt.Hamiltonian(ham)
        d = torch.as_tensor(theta, device="cuda")
        for _ in range(args.steps):
            e, g = c.expect_grad(d, H)
        torch.cuda.synchronize()
        print("rows", args.rows, "plan", c.info(), "E[0]", float(e[0]))
    elif args.workload == "qaoa":
        rng = np.random.default_rng(args.qubits)
        edges = W.random_regular3(args.qubits, rng)
        c = nt.Circuit(W.qaoa_circuit(args.qubits, edges, args.layers), specialize=args.specialize)
        H = nt.Hamiltonian(W.zz_on_edges(args.qubits, edges))
        d = torch.as_tensor(rng.uniform(0, np.pi, size=(args.rows, 2 * args.layers)), device="cuda")
        for _ in range(args.steps):
            e, g = c.expect_grad(d, H)
        torch.cuda.synchronize()
        print("rows", args.rows, "plan", c.info(), "E[0]", float(e[0]))
    elif args.workload == "noisy16":
        circ, n_traj, seed, obs = W.noisy16_workload()
        c = nt.Circuit(circ, specialize=args.specialize)
        for _ in range(args.steps):
            st = c.apply(None, n_traj, seed=seed)
            vals = [c.expect(st, nt.Hamiltonian(o)) for o in obs]
        torch.cuda.synchronize()
        print("trajectories", n_traj, "plan", c.info(), "<Z0>", float(vals[0].mean()))
    elif args.workload == "tn40":
        circ = W.example_block_circuit(40, 6)
        net = nt.CircuitNetwork(circ, {20: 3}, prune=0, split=True, rank_cap=26, greedy_trials=16)
        th = torch.as_tensor(np.random.default_rng(1009).uniform(-1.5, 1.5, (args.rows, circ.n_params))
                             .astype(np.float32), device="cuda")
        for _ in range(args.steps):
            out = net.expect(th, precision=args.precision)
        torch.cuda.synchronize()
        print("rows", args.rows, "info", net.info(), "<Z20>[0]", float(out[0, 0]))
    elif args.workload == "cone200":
        n, gates0, zq = W.brick200_workload()
        lc = nt.LightCone(n, [(a, b) for a, b, _ in gates0], zq, greedy_trials=64)
        lc.set_cluster(args.cluster)
        gl = [gates0] + [W.brickwork_u4(n, 8, np.random.default_rng(s)) for s in range(1, args.rows)]
        g = torch.as_tensor(np.stack([np.stack([u for (_, _, u) in x]) for x in gl]).astype(np.complex64),
                            device="cuda")
        for _ in range(args.steps):
            out = lc.contract(g)
        torch.cuda.synchronize()
        print("rows", args.rows, "info", lc.info(), "<ZZ>[0]", float(out[0, 0]))
    elif args.workload == "hea10_one":
        circ, theta, obs = W.hea10_workload()
        c = nt.Circuit(circ, dtype=nt.TC_C128)
        d = torch.as_tensor(theta, device="cuda")
        o = nt.Observables(obs)
        for _ in range(args.steps):
            st, vals = c.apply_expect(d, o, 1)
        torch.cuda.synchronize()
        print("one launch", vals.cpu().numpy())
    elif args.workload == "qgt":
        circ, theta, _ = W.tfim_workload(args.qubits, 10, args.rows)
        c = nt.Circuit(circ)
        d = torch.as_tensor(theta, device="cuda")
        for _ in range(args.steps):
            g = c.qgt(d)
        torch.cuda.synchronize()
        print("rows", args.rows, "qubits", args.qubits, "QFI_00", float(4 * g[0, 0, 0].real))
    else:
        circ, theta, obs = W.hea10_workload()
        c = nt.Circuit(circ, dtype=nt.TC_C128)
        d = torch.as_tensor(theta, device="cuda")
        for _ in range(args.steps):
            st = c.apply(d, 1)
            vals = [c.expect(st, nt.Hamiltonian(o)) for o in obs]
        torch.cuda.synchronize()
        print("plan", c.info(), [float(v[0]) for v in vals])


if __name__ == "__main__":
    main()
