"""Light-cone reduction of a MaxCut QAOA edge term (test infrastructure).

The oracle evaluates a wide QAOA circuit's energy and gradient edge by edge
on each edge's light cone; this module only selects the gates and qubits of a
cone (no arithmetic of the method).  Pinned against the full-circuit oracle in
tests/test_qaoa_cone_host.py.
"""
from paper_2205_10091_b300 import workloads as W


def edge_cone(circ, u, v):
    """The backward light cone of Z_u Z_v in a circuit of RZZ and RX gates from
    |+>^n.  Walking the gates backwards, S holds the qubits the evolved
    observable acts on and X those it acts on non-diagonally: an RX is kept
    when its qubit is in S (it then joins X), an RZZ when it touches X (its
    qubits then join S).  A skipped gate commutes with the evolved observable
    (an RZZ off X meets only diagonal factors, an RX off S only identities), so
    <Z_u Z_v> of the kept gates on the qubits of S (the others stay |+>) is
    exact."""
    S, X = {u, v}, set()
    keep = []
    for op in reversed(list(circ.ops)):
        k, q0, q1 = int(op["kind"]), int(op["q0"]), int(op["q1"])
        if k == W.OP_RZZ:
            if q0 in X or q1 in X:
                keep.append(op)
                S |= {q0, q1}
        else:
            assert k == W.OP_RX
            if q0 in S:
                keep.append(op)
                X.add(q0)
    keep.reverse()
    qmap = {q: i for i, q in enumerate(sorted(S))}
    b = W.OpBuilder(len(qmap), W.INIT_PLUS)
    for op in keep:
        k, q0, q1 = int(op["kind"]), int(op["q0"]), int(op["q1"])
        if k == W.OP_RZZ:
            b.rzz(qmap[q0], qmap[q1], int(op["param"]), scale=float(op["scale"]))
        else:
            assert k == W.OP_RX
            b.rx(qmap[q0], int(op["param"]), scale=float(op["scale"]))
    return b.build(circ.n_params), W.pauli_sum(len(qmap), [(1.0, {qmap[u]: 3, qmap[v]: 3})])
