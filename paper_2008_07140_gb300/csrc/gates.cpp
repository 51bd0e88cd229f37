// Host gate library (Appendix A-1) and DAGGER / CONTROL block expansion, in FP64.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace qsim {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char *last_error() { return g_err; }

qsim_status cuda_fail(cudaError_t e, const char *what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  if (e == cudaErrorMemoryAllocation) return QSIM_ENOMEM;
  return QSIM_ECUDA;
}

// Matrices of Appendix A-1 (first listed qubit = most significant index bit).
int named_matrix(int kind, const double *p, std::vector<cd> &m) {
  const double r = std::sqrt(0.5);
  const cd I(0.0, 1.0);
  auto one = [&](cd a, cd b, cd c, cd d) {
    m = {a, b, c, d};
    return 1;
  };
  switch (kind) {
    case QSIM_OP_H: return one(r, r, r, -r);
    case QSIM_OP_X: return one(0.0, 1.0, 1.0, 0.0);
    case QSIM_OP_Y: return one(0.0, -I, I, 0.0);
    case QSIM_OP_Z: return one(1.0, 0.0, 0.0, -1.0);
    case QSIM_OP_S: return one(1.0, 0.0, 0.0, I);
    case QSIM_OP_T: return one(1.0, 0.0, 0.0, cd(r, r));
    // principal square roots of X and Y (random-circuit gate set, not in the paper)
    case QSIM_OP_SX: return one(cd(0.5, 0.5), cd(0.5, -0.5), cd(0.5, -0.5), cd(0.5, 0.5));
    case QSIM_OP_SY: return one(cd(0.5, 0.5), cd(-0.5, -0.5), cd(0.5, 0.5), cd(0.5, 0.5));
    case QSIM_OP_RX: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      return one(c, -I * s, -I * s, c);
    }
    case QSIM_OP_RY: {
      double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
      return one(c, -s, s, c);
    }
    case QSIM_OP_RZ: return one(std::exp(-I * (p[0] / 2)), 0.0, 0.0, std::exp(I * (p[0] / 2)));
    case QSIM_OP_U4: {
      double a = p[0], b = p[1], g = p[2], d = p[3];
      double c = std::cos(g / 2), s = std::sin(g / 2);
      return one(std::exp(I * (a - b / 2 - d / 2)) * c, -std::exp(I * (a - b / 2 + d / 2)) * s,
                 std::exp(I * (a + b / 2 - d / 2)) * s, std::exp(I * (a + b / 2 + d / 2)) * c);
    }
    case QSIM_OP_CNOT:
    case QSIM_OP_CZ:
    case QSIM_OP_CR:
    case QSIM_OP_SWAP:
    case QSIM_OP_ISWAP: {
      m.assign(16, 0.0);
      m[0] = m[5] = 1.0;
      if (kind == QSIM_OP_CNOT) {
        m[11] = m[14] = 1.0;
      } else if (kind == QSIM_OP_CZ) {
        m[10] = 1.0;
        m[15] = -1.0;
      } else if (kind == QSIM_OP_CR) {
        m[10] = 1.0;
        m[15] = std::exp(I * p[0]);
      } else {
        m[5] = 0.0;
        m[15] = 1.0;
        cd off = kind == QSIM_OP_SWAP ? cd(1.0) : -I;
        m[6] = m[9] = off;
      }
      return 2;
    }
    case QSIM_OP_TOFFOLI: {
      m.assign(64, 0.0);
      for (int i = 0; i < 6; ++i) m[i * 8 + i] = 1.0;
      m[6 * 8 + 7] = m[7 * 8 + 6] = 1.0;
      return 3;
    }
    default: return -1;
  }
}

// Controlled named gates become (target, controls, 2x2): the paper's CNOT / CZ / CR /
// TOFFOLI matrices are identity except on the block where all controls are 1.
static bool as_controlled(int kind, const int32_t *q, const double *p, Gate &g) {
  const cd I(0.0, 1.0);
  switch (kind) {
    case QSIM_OP_CNOT: g.m = {0.0, 1.0, 1.0, 0.0}; break;
    case QSIM_OP_CZ: g.m = {1.0, 0.0, 0.0, -1.0}; break;
    case QSIM_OP_CR: g.m = {1.0, 0.0, 0.0, std::exp(I * p[0])}; break;
    case QSIM_OP_TOFFOLI: g.m = {0.0, 1.0, 1.0, 0.0}; break;
    default: return false;
  }
  int nctl = kind == QSIM_OP_TOFFOLI ? 2 : 1;
  g.nt = 1;
  for (int j = 0; j < nctl; ++j) g.ctrl.push_back(q[j]);
  g.t[0] = q[nctl];
  return true;
}

namespace {

struct Item {
  int type;  // 0 gate, 1 dagger block, 2 control block
  Gate g;
  std::vector<int> ctl;
  std::vector<Item> inner;
};

qsim_status parse(const qsim_op *ops, size_t nops, size_t &pos, int end_kind, int n,
                  std::vector<Item> &items) {
  while (pos < nops) {
    const qsim_op &op = ops[pos];
    if (op.kind == QSIM_OP_DAGGER || op.kind == QSIM_OP_CONTROL) {
      Item it;
      it.type = op.kind == QSIM_OP_DAGGER ? 1 : 2;
      if (it.type == 2) {
        if (op.nq < 1 || op.nq > 3) {
          set_error("CONTROL needs 1..3 qubits (op %zu)", pos);
          return QSIM_EINVAL;
        }
        for (int j = 0; j < op.nq; ++j) {
          if (op.qubits[j] < 0 || op.qubits[j] >= n) {
            set_error("CONTROL qubit %d out of range (op %zu)", op.qubits[j], pos);
            return QSIM_EINVAL;
          }
          it.ctl.push_back(op.qubits[j]);
        }
      }
      ++pos;
      QS_TRY(parse(ops, nops, pos, it.type == 1 ? QSIM_OP_ENDDAGGER : QSIM_OP_ENDCONTROL, n,
                   it.inner));
      items.push_back(std::move(it));
      continue;
    }
    if (op.kind == QSIM_OP_ENDDAGGER || op.kind == QSIM_OP_ENDCONTROL) {
      if (op.kind != end_kind) {
        set_error("unbalanced block end at op %zu", pos);
        return QSIM_EINVAL;
      }
      ++pos;
      return QSIM_OK;
    }
    Item it;
    it.type = 0;
    Gate &g = it.g;
    g.kind = op.kind;
    if (op.kind == QSIM_OP_MATRIX) {
      if (op.nq < 1 || op.nq > 3 || !op.matrix) {
        set_error("MATRIX op %zu needs 1..3 qubits and a matrix", pos);
        return QSIM_EINVAL;
      }
      int dim = 1 << op.nq;
      g.nt = op.nq;
      g.m.resize((size_t)dim * dim);
      for (int i = 0; i < dim * dim; ++i) g.m[i] = cd(op.matrix[2 * i], op.matrix[2 * i + 1]);
      for (int j = 0; j < op.nq; ++j) g.t[j] = op.qubits[j];
    } else if (!as_controlled(op.kind, op.qubits, op.params, g)) {
      int k = named_matrix(op.kind, op.params, g.m);
      if (k < 0) {
        set_error("unknown op kind %d at op %zu", op.kind, pos);
        return QSIM_EINVAL;
      }
      g.nt = k;
      for (int j = 0; j < k; ++j) g.t[j] = op.qubits[j];
    }
    int expect = op.kind == QSIM_OP_MATRIX ? op.nq : (int)(g.nt + g.ctrl.size());
    if (op.nq != expect) {
      set_error("op %zu (kind %d) lists %d qubits, needs %d", pos, op.kind, op.nq, expect);
      return QSIM_EINVAL;
    }
    if (op.nc < 0 || (op.nc > 0 && !op.controls)) {
      set_error("op %zu: bad controls", pos);
      return QSIM_EINVAL;
    }
    for (int j = 0; j < op.nc; ++j) g.ctrl.push_back(op.controls[j]);
    items.push_back(std::move(it));
    ++pos;
  }
  if (end_kind != -1) {
    set_error("missing block end");
    return QSIM_EINVAL;
  }
  return QSIM_OK;
}

void adjoint(Gate &g) {
  int dim = 1 << g.nt;
  std::vector<cd> a((size_t)dim * dim);
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) a[(size_t)r * dim + c] = std::conj(g.m[(size_t)c * dim + r]);
  g.m.swap(a);
}

// Under an odd number of DAGGERs a block runs backwards with each gate replaced by its
// adjoint; CONTROL adds its qubits to every gate inside.
void flatten(const std::vector<Item> &items, bool dag, std::vector<int> &ctl,
             std::vector<Gate> &out) {
  size_t cnt = items.size();
  for (size_t k = 0; k < cnt; ++k) {
    const Item &it = items[dag ? cnt - 1 - k : k];
    if (it.type == 0) {
      Gate g = it.g;
      if (dag) adjoint(g);
      g.ctrl.insert(g.ctrl.end(), ctl.begin(), ctl.end());
      out.push_back(std::move(g));
    } else if (it.type == 1) {
      flatten(it.inner, !dag, ctl, out);
    } else {
      size_t keep = ctl.size();
      ctl.insert(ctl.end(), it.ctl.begin(), it.ctl.end());
      flatten(it.inner, dag, ctl, out);
      ctl.resize(keep);
    }
  }
}

}  // namespace

qsim_status expand_ops(const qsim_op *ops, size_t nops, int n, std::vector<Gate> &out) {
  if (nops > 0 && !ops) {
    set_error("ops is NULL");
    return QSIM_EINVAL;
  }
  std::vector<Item> items;
  size_t pos = 0;
  QS_TRY(parse(ops, nops, pos, -1, n, items));
  std::vector<int> ctl;
  out.clear();
  flatten(items, false, ctl, out);
  for (size_t i = 0; i < out.size(); ++i) {
    const Gate &g = out[i];
    unsigned long long seen = 0;
    for (int j = 0; j < g.nt + (int)g.ctrl.size(); ++j) {
      int q = j < g.nt ? g.t[j] : g.ctrl[j - g.nt];
      if (q < 0 || q >= n) {
        set_error("gate %zu: qubit %d out of range [0, %d)", i, q, n);
        return QSIM_EINVAL;
      }
      if (seen >> q & 1ULL) {
        set_error("gate %zu: qubit %d listed twice", i, q);
        return QSIM_EINVAL;
      }
      seen |= 1ULL << q;
    }
  }
  return QSIM_OK;
}

}  // namespace qsim
