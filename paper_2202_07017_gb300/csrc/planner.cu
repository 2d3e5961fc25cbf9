// Gate-fusion planner (host, fp64).
//
// The paper applies a circuit gate by gate (Sec. 2, Eq. 1), one pass over
// the 2^n-amplitude state per gate.  Here consecutive gates are grouped
// into passes: a pass stages m amplitude-index bits S (the L lowest bits,
// giving contiguous runs, plus high bits) so that each thread block loads
// one 2^m-amplitude slice into shared memory, applies every gate of the
// pass whose qubits lie in S, and writes the slice back: one HBM round
// trip for many gates.  Gates on disjoint qubits commute, so any order
// that keeps, for every qubit, the circuit order of the gates touching it
// computes the same product.
//
// Planning steps:
//   1. gates become FGates (1-qubit dense with controls, phase on an
//      all-ones subspace, SWAP with controls, or "alone" for anything else
//      or anything wider than fuse_k qubits); consecutive uncontrolled
//      1-qubit gates on one qubit are multiplied into one 2x2 in fp64;
//   2. a pass grows S greedily from the earliest remaining gate, taking
//      every later gate whose qubits fit in S and that no skipped earlier
//      gate overlaps; unused places in S are filled with the lowest free
//      bits (longer contiguous runs);
//   3. the pass's gates are list-scheduled into register groups of at
//      most fuse_k qubits (a gate joins the open group when every earlier
//      unscheduled gate it overlaps is scheduled and the union stays within
//      fuse_k qubits).
#include <algorithm>

#include "sv_internal.cuh"

namespace sv {
namespace {

int popc(uint64_t x) { return __builtin_popcountll(x); }

bool is_zero(cd z) { return z.re == 0.0 && z.im == 0.0; }
bool is_one(cd z) { return z.re == 1.0 && z.im == 0.0; }

// a := b * a (2x2 complex, row-major)
void mul2_left(const cd* b, cd* a) {
  cd r[4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double re = 0, im = 0;
      for (int k = 0; k < 2; ++k) {
        const cd x = b[i * 2 + k], y = a[k * 2 + j];
        re += x.re * y.re - x.im * y.im;
        im += x.re * y.im + x.im * y.re;
      }
      r[i * 2 + j] = {re, im};
    }
  for (int e = 0; e < 4; ++e) a[e] = r[e];
}

// The FGate of circuit gate g (index i) with matrix G, in bit positions.
FGate classify(const sv_gate& g, int i, int n, const HostMatrix& G, int kmax) {
  FGate f;
  f.orig = i;
  f.origs.push_back(i);
  int tp[SV_MAX_TARGETS];
  uint64_t cm = 0;
  for (int j = 0; j < g.n_tar; ++j) {
    tp[j] = n - 1 - g.targets[j];
    f.qmask |= uint64_t(1) << tp[j];
  }
  for (int j = 0; j < g.n_ctrl; ++j) cm |= uint64_t(1) << (n - 1 - g.controls[j]);
  f.qmask |= cm;
  const int k = g.n_tar, d = 1 << k;
  bool diag = true, ones = true;
  for (int r = 0; r < d; ++r)
    for (int q = 0; q < d; ++q)
      if (r != q && !is_zero(G.at(r, q))) diag = false;
  for (int r = 0; r + 1 < d; ++r)
    if (!is_one(G.at(r, r))) ones = false;
  bool swap = k == 2;
  if (swap) {
    static const int perm[4] = {0, 2, 1, 3};
    for (int r = 0; r < 4; ++r)
      for (int q = 0; q < 4; ++q)
        if (q == perm[r] ? !is_one(G.at(r, q)) : !is_zero(G.at(r, q))) swap = false;
  }
  if (diag && ones) {
    f.type = FG_PHASE;
    f.cmask = f.qmask;
    f.m[0] = G.at(d - 1, d - 1);
  } else if (swap) {
    f.type = FG_SWAP;
    f.a = tp[0];
    f.b = tp[1];
    f.cmask = cm;
  } else if (k == 1) {
    f.type = FG_1Q;
    f.t = tp[0];
    f.cmask = cm;
    for (int e = 0; e < 4; ++e) f.m[e] = G.m[e];
  } else {
    f.type = FG_ALONE;
  }
  if (popc(f.qmask) > kmax) f.type = FG_ALONE;
  // a multi-qubit Pauli string runs as one rotation pass of its own
  if (g.kind == SV_GATE_PAULI && k > 1) f.type = FG_ALONE;
  return f;
}

// Appends f, multiplying an uncontrolled 1-qubit gate into the previous
// operation on its qubit when that is an uncontrolled 1-qubit gate.
void push_fgate(FGate f, std::vector<int>* last, std::vector<FGate>* out) {
  if (f.type == FG_1Q && f.cmask == 0) {
    const int p = (*last)[f.t];
    if (p >= 0 && (*out)[p].type == FG_1Q && (*out)[p].cmask == 0 && (*out)[p].t == f.t) {
      mul2_left(f.m, (*out)[p].m);
      for (int o : f.origs) (*out)[p].origs.push_back(o);
      (*out)[p].orig = f.orig;
      return;
    }
  }
  out->push_back(std::move(f));
  for (int b = 0; b < 64; ++b)
    if ((out->back().qmask >> b) & 1) (*last)[b] = (int)out->size() - 1;
}

bool to_fgates(const sv_circuit* c, const double* theta, int kmax, std::vector<FGate>* out) {
  const int n = c->n_qubits;
  std::vector<int> last(64, -1);
  HostMatrix G;
  for (int i = 0; i < c->n_gates; ++i) {
    const sv_gate& g = c->gates[i];
    if (!gate_matrix(g, theta, c->mat_pool, &G)) {
      set_error("gate %d: cannot build matrix", i);
      return false;
    }
    push_fgate(classify(g, i, n, G, kmax), &last, out);
  }
  return true;
}

// 2x2 complex products (row-major)
void mul2(const cd* a, const cd* b, cd* out) {  // out = a b
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double re = 0, im = 0;
      for (int k = 0; k < 2; ++k) {
        const cd x = a[i * 2 + k], y = b[k * 2 + j];
        re += x.re * y.re - x.im * y.im;
        im += x.re * y.im + x.im * y.re;
      }
      out[i * 2 + j] = {re, im};
    }
}

// (a, d, re b, im b) of an FG_GRAD's generator [[a, b], [conj b, d]]
void generator_of(const FGate& g, double* out) {
  static const double kPauli[4][4] = {{0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, -1}, {1, -1, 0, 0}};
  if (g.pauli) {
    for (int e = 0; e < 4; ++e) out[e] = kPauli[g.pauli][e];
  } else {
    out[0] = g.m[0].re;
    out[1] = g.m[3].re;
    out[2] = g.m[1].re;
    out[3] = g.m[1].im;
  }
}

// Reverse sweep over [lo, hi): gate hi-1 first, each as its adjoint, a
// parameterised gate preceded by its FG_GRAD.  Uncontrolled 1-qubit
// adjoints are kept pending per qubit (their product W, not yet applied)
// until another kind of gate touches the qubit; a gradient met while W is
// pending is evaluated on the untransformed states with the generator
// W^dagger P W (Im<W lambda|P|W psi> = Im<lambda|W^dagger P W|psi>), so a
// run RZ, RY, RX on one qubit costs one un-apply.  Gradients on one qubit with
// nothing else touching it in between share one FG_GRAD (up to kGradPerOp):
// the ops between them act on other qubits, commute with the generator and
// leave the inner product unchanged.  A parameterised gate
// wider than kmax stays unfused with its gradient.
bool to_fgates_reverse(const sv_circuit* c, const double* theta, int lo, int hi,
                       const std::vector<int>& slot_of, int kmax, std::vector<FGate>* out) {
  const int n = c->n_qubits;
  std::vector<int> last(64, -1);
  struct Pend {
    bool on = false;
    cd W[4];
    int orig = -1;
    std::vector<int> origs;  // every circuit gate folded into W
  };
  std::vector<Pend> pend(64);
  auto flush = [&](int t) {
    if (!pend[t].on) return;
    FGate f;
    f.type = FG_1Q;
    f.t = t;
    f.qmask = uint64_t(1) << t;
    f.cmask = 0;
    for (int e = 0; e < 4; ++e) f.m[e] = pend[t].W[e];
    f.orig = pend[t].orig;
    f.origs = pend[t].origs;
    push_fgate(std::move(f), &last, out);
    pend[t].on = false;
    pend[t].origs.clear();
  };
  HostMatrix G, D;
  for (int i = hi - 1; i >= lo; --i) {
    const sv_gate& g = c->gates[i];
    if (!gate_matrix(g, theta, c->mat_pool, &G)) {
      set_error("gate %d: cannot build matrix", i);
      return false;
    }
    const int d = 1 << G.k;
    D.k = G.k;
    for (int r = 0; r < d; ++r)
      for (int q = 0; q < d; ++q) {
        const cd z = G.at(q, r);
        D.m[r * d + q] = {z.re, -z.im};
      }
    FGate f = classify(g, i, n, D, kmax);
    if (f.type == FG_PHASE && G.k == 1 && g.n_ctrl == 0) {  // Z, U1: a 1-qubit adjoint too
      f.type = FG_1Q;
      f.t = n - 1 - g.targets[0];
      f.cmask = 0;
      for (int e = 0; e < 4; ++e) f.m[e] = D.m[e];
    }
    // generator of a parameterised gate: 1 X, 2 Y, 3 Z on its target; a
    // multi-qubit PAULI string (4) stays unfused with its own adjoint kernel
    int pauli = 0;
    if (g.param >= 0) {
      if (g.kind == SV_GATE_PAULI)
        pauli = g.n_tar == 1 ? (g.paulis & 3) : 4;
      else
        pauli = g.kind == SV_GATE_RX ? 1 : g.kind == SV_GATE_RY ? 2 : 3;
    }
    if (g.kind == SV_GATE_PAULI && g.n_tar > 1) f.type = FG_ALONE;
    if (f.type == FG_1Q && f.cmask == 0) {
      const int t = f.t;
      if (pauli) {
        FGate gr;
        gr.type = FG_GRAD;
        gr.qmask = uint64_t(1) << t;
        gr.t = t;
        gr.cmask = 0;
        gr.pauli = pauli;
        gr.slot = slot_of[i];
        gr.orig = i;
        if (pend[t].on) {  // generator W^dagger P W, stored as a Hermitian 2x2
          static const cd PX[4] = {{0, 0}, {1, 0}, {1, 0}, {0, 0}};
          static const cd PY[4] = {{0, 0}, {0, -1}, {0, 1}, {0, 0}};
          static const cd PZ[4] = {{1, 0}, {0, 0}, {0, 0}, {-1, 0}};
          const cd* P = pauli == 1 ? PX : pauli == 2 ? PY : PZ;
          const cd* W = pend[t].W;
          const cd Wd[4] = {{W[0].re, -W[0].im}, {W[2].re, -W[2].im},
                            {W[1].re, -W[1].im}, {W[3].re, -W[3].im}};
          cd PW[4], M[4];
          mul2(P, W, PW);
          mul2(Wd, PW, M);
          gr.pauli = 0;  // general generator in m
          for (int e = 0; e < 4; ++e) gr.m[e] = M[e];
        }
        // nothing has touched t since a gradient on t: evaluate this one there
        const int p = last[t];
        if (p >= 0 && (*out)[p].type == FG_GRAD && (*out)[p].cmask == 0 && (*out)[p].t == t &&
            (*out)[p].ng < kGradPerOp) {
          FGate& h = (*out)[p];
          if (h.ng == 1) {
            generator_of(h, h.gen[0]);
            h.gslots[0] = h.slot;
          }
          generator_of(gr, h.gen[h.ng]);
          h.gslots[h.ng++] = gr.slot;
        } else {
          push_fgate(std::move(gr), &last, out);
        }
      }
      if (pend[t].on) {
        cd r[4];
        mul2(f.m, pend[t].W, r);  // this adjoint acts after the pending product
        for (int e = 0; e < 4; ++e) pend[t].W[e] = r[e];
      } else {
        pend[t].on = true;
        for (int e = 0; e < 4; ++e) pend[t].W[e] = f.m[e];
      }
      pend[t].orig = i;
      pend[t].origs.push_back(i);
      continue;
    }
    for (int b = 0; b < 64; ++b)
      if ((f.qmask >> b) & 1) flush(b);
    if (pauli) {
      if (f.type == FG_ALONE) {
        f.pauli = pauli;
        f.slot = slot_of[i];
      } else {
        FGate gr;
        gr.type = FG_GRAD;
        gr.qmask = f.qmask;
        gr.t = n - 1 - g.targets[0];
        gr.cmask = f.qmask & ~(uint64_t(1) << gr.t);
        gr.pauli = pauli;
        gr.slot = slot_of[i];
        gr.orig = i;
        push_fgate(std::move(gr), &last, out);
      }
    }
    push_fgate(std::move(f), &last, out);
  }
  for (int b = 0; b < 64; ++b) flush(b);
  return true;
}

int local_of(const std::vector<int>& S, int bit) {
  return (int)(std::lower_bound(S.begin(), S.end(), bit) - S.begin());
}

}  // namespace

FusionConfig fusion_config(int n, sv_dtype dt, int fuse_k) {
  FusionConfig c;
  c.fuse_k = std::min(fuse_k, 4);  // the pass kernel holds register groups of <= 4 qubits
  int m = std::min(n, dt == SV_C64 ? 13 : 12);
  // keep at least 2^8 blocks for mid-size states, down to 2^10 amplitudes
  if (n > 10) m = std::max(std::min(m, n - 8), std::min(n, 10));
  c.m = m;
  c.L = std::min(dt == SV_C64 ? 5 : 4, m);
  if (c.m - c.L < fuse_k) c.L = std::max(1, c.m - fuse_k);
  return c;
}

FusionConfig fusion_config_reverse(int n, sv_dtype dt, int fuse_k) {
  // two 2^k tiles per thread: up to 4 qubits for complex64, 3 for complex128
  FusionConfig c = fusion_config(n, dt, std::min(fuse_k, dt == SV_C64 ? 4 : 3));
  if (c.m > 10) {
    c.m -= 1;
    if (c.m - c.L < c.fuse_k) c.L = std::max(1, c.m - c.fuse_k);
  }
  return c;
}

namespace {

// Passes (steps 2 and 3 of the planning) over the operation list F.
void form_passes(const std::vector<FGate>& F, int n, const FusionConfig& cfg,
                 std::vector<FusionItem>* out) {
  std::vector<char> done(F.size(), 0);
  const uint64_t lowL = (cfg.L >= 64) ? ~uint64_t(0) : ((uint64_t(1) << cfg.L) - 1);
  size_t first = 0;
  out->clear();
  while (true) {
    while (first < F.size() && done[first]) ++first;
    if (first == F.size()) break;
    const FGate& f0 = F[first];
    if (f0.type == FG_ALONE || popc(f0.qmask & ~lowL) > cfg.m - cfg.L) {
      for (int o : f0.origs) {
        FusionItem it;
        it.gate = o;
        it.pauli = f0.pauli;
        it.slot = f0.slot;
        out->push_back(it);
      }
      done[first] = 1;
      continue;
    }
    // 2. grow S from the earliest remaining gate
    uint64_t S = lowL, blocked = 0;
    int nS = cfg.L, ngrads = 0;
    std::vector<int> take;
    for (size_t j = first; j < F.size(); ++j) {
      if (done[j]) continue;
      const FGate& f = F[j];
      bool ok = f.type != FG_ALONE && !(f.qmask & blocked) && (int)take.size() < cfg.max_ops &&
                (f.type != FG_GRAD || ngrads + f.ng <= cfg.max_grads);
      if (ok) {
        const uint64_t need = f.qmask & ~S;
        if (nS + popc(need) > cfg.m) {
          ok = false;
        } else {
          S |= need;
          nS += popc(need);
        }
      }
      if (ok) {
        take.push_back((int)j);
        if (f.type == FG_GRAD) ngrads += f.ng;
      } else
        blocked |= f.qmask;
    }
    for (int b = 0; b < n && nS < cfg.m; ++b)
      if (!((S >> b) & 1)) {
        S |= uint64_t(1) << b;
        ++nS;
      }
    // 3. register groups by list scheduling
    std::vector<int> pending = take;
    std::vector<FusedGroup> groups;
    std::vector<int> placed;
    std::vector<FusionItem> none;
    FusionItem item;
    item.is_pass = true;
    FusedPass& P = item.pass;
    for (int b = 0; b < n; ++b)
      if ((S >> b) & 1) P.S.push_back(b);
    P.L = 0;
    while (P.L < (int)P.S.size() && P.S[P.L] == P.L) ++P.L;
    while (!pending.empty() && (int)groups.size() < cfg.max_groups) {
      uint64_t gq = F[pending[0]].qmask, acc = 0;
      std::vector<int> members, rest;
      for (int j : pending) {
        const FGate& f = F[j];
        if (!(f.qmask & acc) && popc(gq | f.qmask) <= cfg.fuse_k) {
          gq |= f.qmask;
          members.push_back(j);
        } else {
          acc |= f.qmask;
          rest.push_back(j);
        }
      }
      // pad every group to the same width (one kernel instantiation per
      // pass; padded bits only widen the thread's tile)
      const int width = std::min<int>(cfg.fuse_k, (int)P.S.size());
      for (int b : P.S) {
        if (popc(gq) >= width) break;
        gq |= uint64_t(1) << b;
      }
      FusedGroup grp;
      for (int b = 0; b < n; ++b)
        if ((gq >> b) & 1) grp.bits[grp.k++] = local_of(P.S, b);
      for (int j : members) {
        grp.ops.push_back((int)P.gates.size());
        P.gates.push_back(F[j]);
        placed.push_back(j);
      }
      groups.push_back(grp);
      pending.swap(rest);
    }
    P.groups = groups;
    for (int j : placed) done[j] = 1;
    out->push_back(std::move(item));
  }
}

}  // namespace

bool plan_fusion(const sv_circuit* c, const double* theta, const FusionConfig& cfg,
                 std::vector<FusionItem>* out) {
  std::vector<FGate> F;
  if (!to_fgates(c, theta, std::min(cfg.fuse_k, cfg.m), &F)) return false;
  form_passes(F, c->n_qubits, cfg, out);
  return true;
}

bool plan_fusion_reverse(const sv_circuit* c, const double* theta, int lo, int hi,
                         const std::vector<int>& slot_of, const FusionConfig& cfg,
                         std::vector<FusionItem>* out) {
  std::vector<FGate> F;
  if (!to_fgates_reverse(c, theta, lo, hi, slot_of, std::min(cfg.fuse_k, cfg.m), &F))
    return false;
  form_passes(F, c->n_qubits, cfg, out);
  return true;
}

}  // namespace sv
