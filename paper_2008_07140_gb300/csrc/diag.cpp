// Host side of the merged diagonal sweep: which gates qualify, what their per-gate sweeps
// would move, and the table of products over the qubits a group touches.
//
// A diagonal gate multiplies amplitude x by one diagonal entry of its matrix, chosen by the
// bits of x at its targets (Eq. 2 with a zero off-diagonal), or by 1 when a control bit of
// x is 0. Diagonal gates commute with each other, so a group of them is one diagonal
// operator whose entry for x is the product of the gates' entries; it depends only on the
// bits of x at the group's qubits. The products are formed in double-double arithmetic
// (TwoProduct with FMA, TwoSum), so a table entry equals the exact product of the FP64
// entries to about 2^-100 before it is rounded to the state's format: the merged sweep
// applies the same FP64 gates as the per-gate sweeps, with one rounding per amplitude.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace qsim {

namespace {

struct DD {
  double hi, lo;
};

inline DD fast_two_sum(double a, double b) {
  const double s = a + b;
  return DD{s, b - (s - a)};
}

inline DD two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return DD{s, (a - (s - bb)) + (b - bb)};
}

// a * b for a double-double a and a double b
inline DD mul(const DD &a, double b) {
  const double p = a.hi * b;
  const double e = std::fma(a.hi, b, -p);
  return fast_two_sum(p, std::fma(a.lo, b, e));
}

inline DD add(const DD &a, const DD &b) {
  const DD s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

inline DD neg(const DD &a) { return DD{-a.hi, -a.lo}; }

struct CDD {
  DD re, im;
};

// (a.re + i a.im) (f.re + i f.im)
inline CDD cmul(const CDD &a, const cd &f) {
  return CDD{add(mul(a.re, f.real()), neg(mul(a.im, f.imag()))), add(mul(a.re, f.imag()), mul(a.im, f.real()))};
}

}  // namespace

bool diag_gate(const Gate &g) {
  if (g.nt < 1 || g.nt > 2) return false;
  const int D = 1 << g.nt;
  bool identity = true;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const cd v = g.m[r * D + c];
      if (r != c && v != 0.0) return false;
      if (r == c && v != 1.0) identity = false;
    }
  return !identity;
}

double diag_gate_bytes(const Gate &g, int n, int B) {
  // the per-gate dispatch: a diagonal whose entries are 1 except the last runs as a phase
  // sweep over the amplitudes with every target and control bit set; any other diagonal as
  // a pair or quad sweep over the amplitudes with every control bit set
  const int D = 1 << g.nt;
  bool phase = true;
  for (int r = 0; r + 1 < D; ++r) phase = phase && g.m[r * D + r] == 1.0;
  unsigned long long must = 0;
  for (int c : g.ctrl) must |= 1ULL << c;
  if (phase)
    for (int j = 0; j < g.nt; ++j) must |= 1ULL << g.t[j];
  // a 64-byte segment holds 64 / B amplitudes: bits below log2(64 / B) select inside it
  const unsigned long long inside = (64ULL / (unsigned long long)B) - 1ULL;
  const int sel = __builtin_popcountll(must & ~inside);
  return 2.0 * B * std::ldexp(1.0, n - sel);
}

size_t append_diag_table(std::vector<unsigned char> &buf, const std::vector<const Gate *> &gs, const DiagIdx &d,
                       int dtype, bool split) {
  const int N = 1 << d.nq;
  // each gate in table-index terms: control bits, target bits, its diagonal
  struct Factor {
    unsigned cm;
    int nt, ti[2];
    cd f[4];
  };
  auto index_bit = [&](int q) {
    for (int j = 0; j < d.nq; ++j)
      if (d.pos[j] == q) return j;
    return -1;  // not reached: the group's qubits include every gate's qubits
  };
  std::vector<Factor> fs;
  for (const Gate *g : gs) {
    Factor f{};
    for (int c : g->ctrl) f.cm |= 1u << index_bit(c);
    f.nt = g->nt;
    for (int j = 0; j < g->nt; ++j) f.ti[j] = index_bit(g->t[j]);
    for (int r = 0; r < (1 << g->nt); ++r) f.f[r] = g->m[(size_t)r * (1u << g->nt) + r];
    fs.push_back(f);
  }
  std::vector<CDD> tab((size_t)N);
  for (int i = 0; i < N; ++i) {
    CDD v{DD{1.0, 0.0}, DD{0.0, 0.0}};
    for (const Factor &f : fs) {
      if ((i & f.cm) != f.cm) continue;
      int r = 0;  // t[0] is the most significant bit of the matrix index
      for (int j = 0; j < f.nt; ++j) r = (r << 1) | (i >> f.ti[j] & 1);
      if (f.f[r] != 1.0) v = cmul(v, f.f[r]);
    }
    tab[i] = v;
  }
  while (buf.size() % 16) buf.push_back(0);
  const size_t off = buf.size();
  if (split) {
    buf.resize(off + (size_t)N * 24);
    float *f = reinterpret_cast<float *>(buf.data() + off);
    for (int i = 0; i < N; ++i) {
      // three floats per part: hi, the rounding residue of hi, and the residue of that
      auto three = [](const DD &x, float &h, float &l, float &t) {
        h = (float)x.hi;
        const double r = (x.hi - (double)h) + x.lo;
        l = (float)r;
        t = (float)(r - (double)l);
      };
      float rh, rl, r3, ih, il, i3;
      three(tab[i].re, rh, rl, r3);
      three(tab[i].im, ih, il, i3);
      const float e[6] = {rh, rl, ih, il, r3, i3};
      memcpy(f + 6 * i, e, sizeof(e));
    }
  } else if (dtype == QSIM_C128) {
    buf.resize(off + (size_t)N * 16);
    double *f = reinterpret_cast<double *>(buf.data() + off);
    for (int i = 0; i < N; ++i) {
      f[2 * i] = tab[i].re.hi + tab[i].re.lo;
      f[2 * i + 1] = tab[i].im.hi + tab[i].im.lo;
    }
  } else {
    buf.resize(off + (size_t)N * 16);
    float *f = reinterpret_cast<float *>(buf.data() + off);
    for (int i = 0; i < N; ++i) {
      const double re = tab[i].re.hi + tab[i].re.lo, im = tab[i].im.hi + tab[i].im.lo;
      f[4 * i] = (float)re;
      f[4 * i + 1] = (float)im;
      f[4 * i + 2] = (float)(re - (double)f[4 * i]);
      f[4 * i + 3] = (float)(im - (double)f[4 * i + 1]);
    }
  }
  return off;
}

}  // namespace qsim
