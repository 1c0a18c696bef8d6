"""Small, self-contained cases for ncu captures.

    python -m paper_2205_10091_b300.profile_case --rows 32            # TFIM-20 x10 energy+gradient
    python -m paper_2205_10091_b300.profile_case --workload noisy16   # 16-qubit noisy trajectories
    python -m paper_2205_10091_b300.profile_case --workload hea10     # 10-qubit complex128 ansatz
    python -m paper_2205_10091_b300.profile_case --workload qgt --qubits 16 --rows 1
                                                          # geometric tensor of the TFIM ansatz (10 layers)
"""
import argparse

import torch

from . import native as nt
from . import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="tfim20", choices=["tfim20", "noisy16", "hea10", "qgt"])
    ap.add_argument("--rows", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--qubits", type=int, default=16)
    args = ap.parse_args()
    if args.workload == "tfim20":
        circ, theta, ham = W.tfim_workload(20, 10, args.rows)
        c = nt.Circuit(circ)
        H = nt.Hamiltonian(ham)
        d = torch.as_tensor(theta, device="cuda")
        for _ in range(args.steps):
            e, g = c.expect_grad(d, H)
        torch.cuda.synchronize()
        print("rows", args.rows, "plan", c.info(), "E[0]", float(e[0]))
    elif args.workload == "noisy16":
        circ, n_traj, seed, obs = W.noisy16_workload()
        c = nt.Circuit(circ)
        for _ in range(args.steps):
            st = c.apply(None, n_traj, seed=seed)
            vals = [c.expect(st, nt.Hamiltonian(o)) for o in obs]
        torch.cuda.synchronize()
        print("trajectories", n_traj, "plan", c.info(), "<Z0>", float(vals[0].mean()))
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
