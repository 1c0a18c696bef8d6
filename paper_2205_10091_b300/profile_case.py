"""One energy+gradient step of the TFIM-20 x 10-layer workload at a chosen
number of rows: a small, self-contained case for ncu captures.

    python -m paper_2205_10091_b300.profile_case --rows 32
"""
import argparse

import torch

from . import native as nt
from . import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1)
    args = ap.parse_args()
    circ, theta, ham = W.tfim_workload(20, 10, args.rows)
    c = nt.Circuit(circ)
    H = nt.Hamiltonian(ham)
    d = torch.as_tensor(theta, device="cuda")
    for _ in range(args.steps):
        e, g = c.expect_grad(d, H)
    torch.cuda.synchronize()
    print("rows", args.rows, "plan", c.info(), "E[0]", float(e[0]))


if __name__ == "__main__":
    main()
