// Density-matrix circuits on the vectorised state |rho>> = sum_xy rho_xy |x>|y>
// (Section "Density matrix simulator"): a 2n-qubit state whose first n
// qubits carry the row index x and the last n the column index y.
//   U rho U^dagger  ->  U on qubit q and conj(U) on qubit n + q
//   Pauli channel rho -> (1-px-py-pz) rho + px X rho X + py Y rho Y + pz Z rho Z
//                   ->  the 4x4 superoperator
//                       (1-p) I(x)I + px X(x)X - py Y(x)Y + pz Z(x)Z on (q, n + q)
//                       (conj(Y) = -Y), applied exactly instead of sampled.
#include <cmath>
#include <string>
#include <vector>

#include "dm.h"

namespace tcb {

namespace {
const double kX[4][2] = {{0, 0}, {1, 0}, {1, 0}, {0, 0}};
const double kY[4][2] = {{0, 0}, {0, -1}, {0, 1}, {0, 0}};
const double kZ[4][2] = {{1, 0}, {0, 0}, {0, 0}, {-1, 0}};
}  // namespace

bool build_dm_ops(int n, const tc_op* ops, int n_ops, const double* pool, int n_pool, std::vector<tc_op>& out,
                  std::vector<double>& out_pool, std::string& err) {
  out.clear();
  out_pool.assign(pool, pool + 2 * (size_t)n_pool);
  auto add_conj = [&](int off, int entries) {
    const int at = (int)(out_pool.size() / 2);
    for (int e = 0; e < entries; ++e) {
      out_pool.push_back(pool[2 * (off + e)]);
      out_pool.push_back(-pool[2 * (off + e) + 1]);
    }
    return at;
  };
  for (int i = 0; i < n_ops; ++i) {
    const tc_op& o = ops[i];
    const bool two = o.kind == TC_OP_RZZ || o.kind == TC_OP_CNOT || o.kind == TC_OP_CZ || o.kind == TC_OP_U2;
    if (o.q0 < 0 || o.q0 >= n || (two && (o.q1 < 0 || o.q1 >= n))) {
      err = "op " + std::to_string(i) + ": qubit out of range";
      return false;
    }
    tc_op a = o, b = o;  // a on the row register, b on the column register
    b.q0 = o.q0 + n;
    b.q1 = two ? o.q1 + n : -1;
    switch (o.kind) {
      case TC_OP_H:
      case TC_OP_X:
      case TC_OP_RY:
      case TC_OP_CNOT:
      case TC_OP_CZ:
        break;  // real matrices: conj(U) = U
      case TC_OP_RX:
      case TC_OP_RZ:
      case TC_OP_RZZ:
        b.scale = -o.scale;  // conj(exp(-i a G / 2)) = exp(+i a G / 2) for G = X, Z, ZZ
        break;
      case TC_OP_U1:
      case TC_OP_U2: {
        const int entries = o.kind == TC_OP_U1 ? 4 : 16;
        if (o.mat < 0 || o.mat + entries > n_pool) {
          err = "op " + std::to_string(i) + ": matrix offset out of range";
          return false;
        }
        b.mat = add_conj(o.mat, entries);
      } break;
      case TC_OP_PAULI_NOISE: {
        const double px = o.px, py = o.py, pz = o.pz, pi = 1.0 - px - py - pz;
        if (!(px >= 0 && py >= 0 && pz >= 0 && pi >= -1e-12)) {
          err = "op " + std::to_string(i) + ": Pauli probabilities outside [0, 1]";
          return false;
        }
        tc_op s{};
        s.kind = TC_OP_U2;
        s.q0 = o.q0;
        s.q1 = o.q0 + n;
        s.param = -1;
        s.scale = 1.0;
        s.mat = (int)(out_pool.size() / 2);
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            // kron(A, B)[2a + b][2c + d] = A[a][c] B[b][d] with A on q, B on n + q
            const int a0 = r >> 1, b0 = r & 1, c0 = c >> 1, d0 = c & 1;
            auto kr = [&](const double (*A)[2], const double (*B)[2]) {
              const double* x = A[a0 * 2 + c0];
              const double* y = B[b0 * 2 + d0];
              return std::pair<double, double>(x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0]);
            };
            double re = (r == c) ? pi : 0.0, im = 0.0;
            auto add = [&](double w, std::pair<double, double> v) {
              re += w * v.first;
              im += w * v.second;
            };
            add(px, kr(kX, kX));
            add(-py, kr(kY, kY));
            add(pz, kr(kZ, kZ));
            out_pool.push_back(re);
            out_pool.push_back(im);
          }
        out.push_back(s);
        continue;
      }
      case TC_OP_RSEL:
        err = "op " + std::to_string(i) + ": random-axis rotations draw per row; not a density-matrix op";
        return false;
      default:
        err = "op " + std::to_string(i) + ": unknown kind";
        return false;
    }
    out.push_back(a);
    out.push_back(b);
  }
  return true;
}

bool build_dm_terms(int n, const uint8_t* structures, const double* weights, int T, std::vector<DmTerm>& out,
                    std::string& err) {
  out.clear();
  for (int t = 0; t < T; ++t) {
    DmTerm d{};
    int ny = 0;
    for (int q = 0; q < n; ++q) {
      const uint8_t c = structures[(size_t)t * n + q];
      if (c > 3) {
        err = "structure entry outside {0,1,2,3} in term " + std::to_string(t);
        return false;
      }
      const uint32_t bit = 1u << (n - 1 - q);
      if (c == 1 || c == 2) d.f |= bit;
      if (c == 2 || c == 3) d.sm |= bit;
      if (c == 2) ++ny;
    }
    d.ny = ny & 3;
    d.w = weights[t];
    if (!std::isfinite(d.w)) {
      err = "weight not finite in term " + std::to_string(t);
      return false;
    }
    out.push_back(d);
  }
  return true;
}

}  // namespace tcb
