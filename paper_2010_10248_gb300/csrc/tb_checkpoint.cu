// Binomial checkpoint schedule for the adjoint-state gradient (the FWI/RTM
// use of the propagator motivated in Sec. I): Griewank's reversal of a chain
// of time steps with a fixed number of stored states.  Host code only.
//
// Model.  X_n = (u^n, u^{n-1}) is the forward state after n steps (X_0 is the
// zero initial condition of Eq. 1 and costs no storage).  The forward step F_n
// maps X_n to X_{n+1}.  Reversing step n (adjoint step k = n + 1) needs
// u^{n+1}, u^n and u^{n-1}: the state X_n plus one evaluation of F_n, which
// the reverse action performs itself.  With s free slots and X_{i0} held, the
// steps i0 .. i0 + l - 1 are reversed by
//   l = 1:  reverse i0;
//   s = 0:  for j = l-1 .. 1: advance X_{i0} -> X_{i0+j}, reverse i0 + j;
//           then reverse i0;
//   else:   advance X_{i0} -> X_{i0+m} into a new slot, reverse the upper
//           l - m steps with s - 1 slots, free the slot, reverse the lower m
//           steps with s slots,
// with the split m that minimises the advanced steps.  The minimum number of
// advanced steps for (l, s) is t l - C(s + t + 1, t - 1), t the smallest
// integer with C(s + 1 + t, t) >= l (the binomial bound of Griewank and
// Walther with the held state counted as one of the s + 1 checkpoints), and
// l (l - 1) / 2 for s = 0.
#include <cstdint>
#include <vector>

#include "tb.h"
#include "tb_internal.cuh"

namespace tbi {

// C(n, k) in double (exact for the sizes used here)
static double binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0.0;
  if (k > n - k) k = n - k;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// advanced steps of the optimal reversal of l steps with s free slots
static double advance_cost(int64_t l, int s) {
  if (l <= 1) return 0.0;
  if (s <= 0) return 0.5 * (double)l * (double)(l - 1);
  const int c = s + 1;  // checkpoints, the held state included
  int t = 0;
  while (binom(c + t, t) < (double)l) ++t;
  return (double)t * (double)l - binom(c + 1 + t - 1, t - 1);
}

namespace {
struct Planner {
  std::vector<CkptAction>* out;
  int S;
  std::vector<char> used;
  int alloc() {
    for (int i = 0; i < S; ++i)
      if (!used[i]) {
        used[i] = 1;
        return i;
      }
    return -3;  // cannot happen: the recursion takes at most S slots
  }
  void rev(int i0, int l, int s, int src) {
    if (l <= 0) return;
    if (l == 1) {
      out->push_back({kCkptReverse, i0, i0, src, src});
      return;
    }
    if (s == 0) {
      for (int j = l - 1; j >= 1; --j) {
        out->push_back({kCkptAdvance, i0, i0 + j, src, kCkptWork});
        out->push_back({kCkptReverse, i0 + j, i0 + j, kCkptWork, kCkptWork});
      }
      out->push_back({kCkptReverse, i0, i0, src, src});
      return;
    }
    int best = 1;
    double bc = 1e300;
    for (int m = 1; m < l; ++m) {
      const double c = m + advance_cost(l - m, s - 1) + advance_cost(m, s);
      if (c < bc) {
        bc = c;
        best = m;
      }
    }
    const int slot = alloc();
    out->push_back({kCkptAdvance, i0, i0 + best, src, slot});
    rev(i0 + best, l - best, s - 1, slot);
    used[slot] = 0;
    rev(i0, best, s, src);
  }
};
}  // namespace

int plan_binomial(int nt, int S, std::vector<CkptAction>* out, int64_t* forward_steps) {
  out->clear();
  if (nt < 1 || S < 0) return TB_EINVAL;
  Planner p{out, S, std::vector<char>(S > 0 ? S : 1, 0)};
  p.rev(0, nt, S, kCkptZero);
  int64_t f = 0;
  for (const CkptAction& a : *out) f += a.kind == kCkptAdvance ? (int64_t)(a.to - a.from) : 1;
  if (forward_steps) *forward_steps = f;
  return TB_OK;
}

}  // namespace tbi

extern "C" int tb_plan_checkpoints(int nt, int n_snapshots, int* actions, int max_actions,
                                   int64_t* forward_steps) {
  std::vector<tbi::CkptAction> v;
  if (nt < 1 || n_snapshots < 0 || n_snapshots > 4096 || max_actions < 0 || (max_actions > 0 && !actions))
    return -TB_EINVAL;
  if (tbi::plan_binomial(nt, n_snapshots, &v, forward_steps) != TB_OK) return -TB_EINVAL;
  for (size_t i = 0; i < v.size() && (int)i < max_actions; ++i) {
    actions[5 * i + 0] = v[i].kind;
    actions[5 * i + 1] = v[i].from;
    actions[5 * i + 2] = v[i].to;
    actions[5 * i + 3] = v[i].src;
    actions[5 * i + 4] = v[i].dst;
  }
  return (int)v.size();
}
