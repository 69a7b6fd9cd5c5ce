// Sweep schedule of one time step: the serial two-site sweep (Sec. III A,
// Fig. 2, App. A) and the Stoudenmire-White segment scheme (Sec. III B,
// Figs. 6-7, App. B). The activity diagrams of App. B are not available as
// text, so the rules are a reading of the prose:
//   * segment k sweeps right in the first half iff k and p/2 have the same
//     parity (the central pair sweeps away from the centre, neighbours
//     alternate); all directions reverse in the second half;
//   * the pair straddling a boundary is updated by the left segment (Sec. III B),
//     which builds both environments next to the boundary afterwards;
//   * turning pairs where the first half ends (a chain end, or a boundary
//     where two sweeps meet) are evolved once by dt when merging is on
//     (App. A); pairs where the first half starts get dt/2 at the start of
//     the first half and dt/2 at the end of the second;
//   * a segment leaving a boundary starts with the one-site step of its
//     boundary site; otherwise two-site and one-site steps alternate as in
//     the serial sweep.
// Ops get stages as soon as their segment's previous op and any
// cross-segment wait allow; one stage runs as one batched launch sequence.
#include <algorithm>
#include <map>

#include "common.h"

namespace tdvp {

static bool right_first(int k, int p) { return (k % 2) == ((p / 2) % 2); }

void build_half(int N, const std::vector<int>& seg_len, int half, int merge,
                std::vector<SchedOp>& out) {
  const int p = (int)seg_len.size();
  std::vector<std::pair<int, int>> b(p);
  int s0 = 0;
  for (int k = 0; k < p; ++k) {
    if (seg_len[k] < 2) fail(TDVP_EINVAL, "every segment needs at least two sites");
    b[k] = {s0, s0 + seg_len[k] - 1};
    s0 += seg_len[k];
  }
  if (s0 != N) fail(TDVP_EINVAL, "segment lengths do not add up to N");
  const int turn = (half == 1 && merge) ? 2 : 1;
  const int ENV_L = 1, ENV_R = 2;
  std::vector<std::vector<SchedOp>> q(p);
  std::map<int, int> start_boundary;  // seg -> index of its start-of-half boundary op
  std::map<int, int> end_boundary;    // seg -> index of its end-of-half boundary op
  auto fwd = [](int k, int j, int tf, int env, int bnd) { return SchedOp{k, 0, j, tf, env, bnd, -1}; };
  auto bck = [](int k, int j) { return SchedOp{k, 1, j, 1, 0, 0, -1}; };
  for (int k = 0; k < p; ++k) {
    const int s = b[k].first, e = b[k].second;
    bool right = right_first(k, p);
    if (half == 2) right = !right;
    auto& Q = q[k];
    if (right) {
      int first_back;
      if (s == 0) {
        if (half == 1 || !merge) Q.push_back(fwd(k, 0, 1, ENV_L, 0));
        first_back = 1;
      } else {
        first_back = s;
      }
      for (int j = first_back; j < e; ++j) {
        Q.push_back(bck(k, j));
        bool last = (j == e - 1) && (e == N - 1);
        Q.push_back(fwd(k, j, last ? turn : 1, last ? ENV_R : ENV_L, 0));
      }
      if (e < N - 1) {
        Q.push_back(bck(k, e));
        Q.push_back(fwd(k, e, turn, ENV_L | ENV_R, 1));
        end_boundary[k] = (int)Q.size() - 1;
      }
    } else {
      int first_back;
      if (e == N - 1) {
        if (half == 1 || !merge) Q.push_back(fwd(k, N - 2, 1, ENV_R, 0));
        first_back = N - 2;
      } else {
        if (half == 1 || !merge) {
          Q.push_back(fwd(k, e, 1, ENV_L | ENV_R, 1));
          start_boundary[k] = (int)Q.size() - 1;
        }
        first_back = e;
      }
      for (int j = first_back; j > s; --j) {
        Q.push_back(bck(k, j));
        bool last = (j - 1 == s) && (s == 0);
        Q.push_back(fwd(k, j - 1, last ? turn : 1, last ? ENV_L : ENV_R, 0));
      }
      if (s > 0) Q.push_back(bck(k, s));
    }
  }
  // as-soon-as-possible stages, iterated to a fixed point
  bool changed = true;
  while (changed) {
    changed = false;
    for (int k = 0; k < p; ++k) {
      int prev = -1;
      for (size_t i = 0; i < q[k].size(); ++i) {
        int st = prev + 1;
        if (i == 0 && start_boundary.count(k - 1))
          st = std::max(st, q[k - 1][start_boundary[k - 1]].stage + 1);
        auto eb = end_boundary.find(k);
        if (eb != end_boundary.end() && (int)i == eb->second)
          st = std::max(st, q[k + 1].back().stage + 1);
        if (st != q[k][i].stage) {
          q[k][i].stage = st;
          changed = true;
        }
        prev = q[k][i].stage;
      }
    }
  }
  out.clear();
  for (int k = 0; k < p; ++k)
    for (auto& o : q[k]) out.push_back(o);
  std::stable_sort(out.begin(), out.end(), [](const SchedOp& a, const SchedOp& c) {
    return a.stage != c.stage ? a.stage < c.stage : a.seg < c.seg;
  });
}

}  // namespace tdvp

namespace tdvp {

// Segmented one-site time step (the paper's outlook on a parallel one-site
// TDVP, read as the one-site sweep inside every segment with the two-site
// scheme's boundary pairs): op kinds 0 = one-site forward step on site j,
// 1 = bond j evolved backward with the centre moving right (site j split,
// its bond matrix carried into site j + 1), 2 = bond j - 1 evolved backward
// with the centre moving left (site j split, carried into site j - 1),
// 3 = the boundary pair (j, j + 1) evolved forward and split back at the
// bond's current dimension. Directions, waits and turning rules are those of
// build_half; a boundary site has its forward step inside the pair step, so a
// segment leaving a boundary starts with the bond next to it. One segment
// gives the serial one-site sweep.
void build_half1(int N, const std::vector<int>& seg_len, int half, int merge, std::vector<SchedOp>& out) {
  const int p = (int)seg_len.size();
  std::vector<std::pair<int, int>> b(p);
  int s0 = 0;
  for (int k = 0; k < p; ++k) {
    if (seg_len[k] < 2) fail(TDVP_EINVAL, "every segment needs at least two sites");
    b[k] = {s0, s0 + seg_len[k] - 1};
    s0 += seg_len[k];
  }
  if (s0 != N) fail(TDVP_EINVAL, "segment lengths do not add up to N");
  const int turn = (half == 1 && merge) ? 2 : 1;
  std::vector<std::vector<SchedOp>> q(p);
  std::map<int, int> start_boundary, end_boundary;
  auto op = [](int k, int kind, int j, int tf) { return SchedOp{k, kind, j, tf, 0, kind == 3 ? 1 : 0, -1}; };
  for (int k = 0; k < p; ++k) {
    const int s = b[k].first, e = b[k].second;
    bool right = right_first(k, p);
    if (half == 2) right = !right;
    auto& Q = q[k];
    if (right) {
      if (s == 0 && (half == 1 || !merge)) Q.push_back(op(k, 0, 0, 1));
      const int last_site = e == N - 1 ? e : e - 1;
      for (int j = s; j < e; ++j) {
        Q.push_back(op(k, 1, j, 1));
        if (j + 1 <= last_site) Q.push_back(op(k, 0, j + 1, (j + 1 == e && e == N - 1) ? turn : 1));
      }
      if (e < N - 1) {
        Q.push_back(op(k, 3, e, turn));
        end_boundary[k] = (int)Q.size() - 1;
      }
    } else {
      if (e == N - 1) {
        if (half == 1 || !merge) Q.push_back(op(k, 0, N - 1, 1));
      } else if (half == 1 || !merge) {
        Q.push_back(op(k, 3, e, 1));
        start_boundary[k] = (int)Q.size() - 1;
      }
      const int first_site = s == 0 ? s : s + 1;
      for (int j = e; j > s; --j) {
        Q.push_back(op(k, 2, j, 1));
        if (j - 1 >= first_site) Q.push_back(op(k, 0, j - 1, (j - 1 == s && s == 0) ? turn : 1));
      }
    }
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int k = 0; k < p; ++k) {
      int prev = -1;
      for (size_t i = 0; i < q[k].size(); ++i) {
        int st = prev + 1;
        if (i == 0 && start_boundary.count(k - 1))
          st = std::max(st, q[k - 1][start_boundary[k - 1]].stage + 1);
        auto eb = end_boundary.find(k);
        if (eb != end_boundary.end() && (int)i == eb->second) st = std::max(st, q[k + 1].back().stage + 1);
        if (st != q[k][i].stage) {
          q[k][i].stage = st;
          changed = true;
        }
        prev = q[k][i].stage;
      }
    }
  }
  out.clear();
  for (int k = 0; k < p; ++k)
    for (auto& o : q[k]) out.push_back(o);
  std::stable_sort(out.begin(), out.end(), [](const SchedOp& a, const SchedOp& c) {
    return a.stage != c.stage ? a.stage < c.stage : a.seg < c.seg;
  });
}

}  // namespace tdvp

namespace tdvp {

// Messages of one half step when the segments are spread over ranks (one GPU
// each; the layout of the paper's Sec. III B: contiguous groups of segments
// per rank). Every cross-segment read of the schedule happens at a boundary
// update, executed by the left segment: before it the right rank sends its
// current Psi_{e+1} and gamma_{e+1} to the left rank; after it the left rank
// sends the new Psi_{e+1}, V_e and beta_{e+1} back (Sec. III B: O(chi^2 (m +
// d)) numbers per boundary). Boundaries inside a rank exchange nothing. With
// the ranks running the stages in lockstep this reproduces the one-rank
// result: the right segment's last op of the half comes in an earlier stage
// than the boundary update, and its next op in a later one.
void exchange_plan(int N, const std::vector<int>& seg_len, const std::vector<int>& seg_rank, int scheme,
                   int merge, int half, std::vector<ExchangeMsg>& out) {
  if (seg_rank.size() != seg_len.size()) fail(TDVP_EINVAL, "one rank per segment");
  std::vector<SchedOp> ops;
  if (scheme == 2) build_half(N, seg_len, half, merge, ops);
  else if (scheme == 1) build_half1(N, seg_len, half, merge, ops);
  else fail(TDVP_EINVAL, "scheme must be 1 (one-site) or 2 (two-site)");
  out.clear();
  for (const SchedOp& o : ops) {
    if (!o.boundary) continue;
    const int left = seg_rank[o.seg], right = seg_rank[o.seg + 1];
    if (left == right) continue;
    const int e = o.j;
    out.push_back(ExchangeMsg{o.stage, 0, right, left, XCH_PSI, e + 1});
    out.push_back(ExchangeMsg{o.stage, 0, right, left, XCH_GAMMA, e + 1});
    out.push_back(ExchangeMsg{o.stage, 1, left, right, XCH_PSI, e + 1});
    out.push_back(ExchangeMsg{o.stage, 1, left, right, XCH_V, e});
    out.push_back(ExchangeMsg{o.stage, 1, left, right, XCH_BETA, e + 1});
  }
}

}  // namespace tdvp
