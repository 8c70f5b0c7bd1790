// Pebble-game search for the memory schedules of one Winograd level
// (Section 4).
//
// The game is played on the values of one level of Winograd's algorithm
// (Section 2) and the blocks that can hold them: the quadrants A11 ... C22
// of the caller's matrices and up to three temporaries.  Section 4's rules
// map to moves as follows.
//   * rules 0 and 3 (compute a value into a new block): a block addition, a
//     recursive product, or a recursive accumulation writes a value into any
//     block; whatever the block held is gone;
//   * rule 2 (compute in place): the same move with the destination equal to
//     the block of an operand;
//   * rule 1 (free a block): implicit, a block whose value is no longer
//     needed may be overwritten;
//   * rule 4 (duplicate a pebble): a copy row.
// A recursive call follows the contract of its kind (which operand blocks it
// overwrites, whether it accumulates into its destination); its destination
// never aliases an operand.  Each of the seven products is computed once.
//
// Values are vectors over three bases: the blocks of A, the blocks of B, and
// the products P1..P7 with the blocks of the input C (coefficients u + v
// beta).  The candidate values are the Section 2 values and, for C <- alpha
// AB + beta C, the intermediate values the accumulating tables (2, 6-9) hold;
// every linear relation among candidates of the allowed forms is a way to
// compute one, so associativity ("U3 = P1 + P6 + P7 in any order") is
// explored as Section 4 describes.
//
// The search is depth first over game states with a visited set keyed by a
// 128-bit fingerprint of the state (temporaries are interchangeable, so
// their contents are sorted first).  A state is pruned as soon as some
// result can no longer be obtained (a value it needs was overwritten and
// cannot be computed again), a block that must be preserved is lost, or an
// admissible bound (rows, block additions, input blocks overwritten) shows
// that the spec's limits cannot be met from it.  The order in which values
// are tried (list order, results first, or both in turn with growing
// budgets) changes what is found first, never whether a schedule exists.
#include "swmm.h"
#include "swmm_search.h"
#include "schedules.h"

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

// ------------------------------------------------------------------ values
enum Space : int8_t { SP_A = 0, SP_B = 1, SP_C = 2 };
constexpr int kDim = 11;  // C space: P1..P7, C11, C12, C21, C22
constexpr size_t kMaxNodes = 64;

struct Vec {
  Space sp = SP_A;
  int8_t u[kDim] = {}, v[kDim] = {};  // coefficient of basis j: u[j] + v[j] beta
  bool operator==(const Vec &o) const {
    return sp == o.sp && !memcmp(u, o.u, kDim) && !memcmp(v, o.v, kDim);
  }
};

// Coefficients c of "u + c v"; beta multiplies only a vector free of beta.
bool scaled(const Vec &x, int coef, Vec *out) {
  *out = x;
  switch (coef) {
    case SWMM_COEF_ONE:
      return true;
    case SWMM_COEF_NEG:
      for (int j = 0; j < kDim; ++j) out->u[j] = -x.u[j], out->v[j] = -x.v[j];
      return true;
    default: {
      const int s = coef == SWMM_COEF_BETA ? 1 : -1;
      for (int j = 0; j < kDim; ++j) {
        if (x.v[j]) return false;
        out->u[j] = 0;
        out->v[j] = (int8_t)(s * x.u[j]);
      }
      return true;
    }
  }
}

Vec add(const Vec &a, const Vec &b) {
  Vec r = a;
  for (int j = 0; j < kDim; ++j) r.u[j] += b.u[j], r.v[j] += b.v[j];
  return r;
}

// Parse "A21+A22", "P5+bC12-bC21", ...: signed terms, 'b' = beta.
bool parse(const char *s, Vec *out) {
  Vec r;
  bool first = true, have_space = false;
  while (*s) {
    int sign = 1;
    if (*s == '+' || *s == '-') {
      sign = *s == '-' ? -1 : 1;
      ++s;
    } else if (!first) {
      return false;
    }
    first = false;
    bool beta = false;
    if (*s == 'b') beta = true, ++s;
    const char m = *s++;
    Space sp;
    int idx;
    if (m == 'A' || m == 'B') {
      if (s[0] < '1' || s[0] > '2' || s[1] < '1' || s[1] > '2') return false;
      sp = m == 'A' ? SP_A : SP_B;
      idx = 2 * (s[0] - '1') + (s[1] - '1');
      s += 2;
    } else if (m == 'C') {
      if (s[0] < '1' || s[0] > '2' || s[1] < '1' || s[1] > '2') return false;
      sp = SP_C;
      idx = 7 + 2 * (s[0] - '1') + (s[1] - '1');
      s += 2;
    } else if (m == 'P') {
      if (*s < '1' || *s > '7') return false;
      sp = SP_C;
      idx = *s - '1';
      s += 1;
    } else {
      return false;
    }
    if (have_space && sp != r.sp) return false;
    r.sp = sp;
    have_space = true;
    (beta ? r.v : r.u)[idx] += (int8_t)sign;
  }
  *out = r;
  return have_space;
}

// ------------------------------------------------------------------- graph
enum DType : int8_t { D_ADD, D_MUL, D_ACC };
struct Deriv {
  DType type;
  int8_t u, v;   // ADD: w = u + coef v; ACC: v is the accumulated value
  int8_t coef;   // SWMM_COEF_*
  int8_t prod;   // MUL / ACC: product index 0..6
  int8_t sign;   // ACC: w = sign P + coef v
  uint64_t rd;   // values it reads
};

struct Node {
  std::string name;
  Vec vec;
  int home = -1;   // inputs: the block holding it on entry; results: the block it must end in
  bool input = false, result = false;
  std::vector<Deriv> der;
  uint64_t need_any = 0;  // values some derivation of it reads
  unsigned finishers = 0; // products an accumulation into it can use (bit p)
};

struct Graph {
  int accumulate = 0;
  std::vector<Node> nodes;
  int prod_a[7], prod_b[7];  // operand values of P1..P7
  uint64_t inputs = 0, results = 0;
};

// Section 2: S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
// T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21; P1 = A11 B11,
// P2 = A12 B21, P3 = S4 B22, P4 = A22 T4, P5 = S1 T1, P6 = S2 T2, P7 = S3 T3;
// U1 = P1 + P2, U2 = P1 + P6, U3 = U2 + P7, U4 = U2 + P5, U5 = U4 + P3,
// U6 = U3 - P4, U7 = U3 + P5 with C = [U1 U5; U6 U7].
struct Def {
  const char *name, *expr;
};
const Def kAB[] = {
    {"A11", "A11"}, {"A12", "A12"}, {"A21", "A21"}, {"A22", "A22"},
    {"B11", "B11"}, {"B12", "B12"}, {"B21", "B21"}, {"B22", "B22"},
    {"S1", "A21+A22"}, {"S2", "A21+A22-A11"}, {"S3", "A11-A21"}, {"S4", "A12-A21-A22+A11"},
    {"T1", "B12-B11"}, {"T2", "B22-B12+B11"}, {"T3", "B22-B12"}, {"T4", "B22-B12+B11-B21"},
    {"P1", "P1"}, {"P2", "P2"}, {"P3", "P3"}, {"P4", "P4"}, {"P5", "P5"}, {"P6", "P6"}, {"P7", "P7"},
    {"U2", "P1+P6"}, {"U3", "P1+P6+P7"}, {"U4", "P1+P6+P5"},
};
const Def kResultsAB[] = {{"U1", "P1+P2"}, {"U5", "P1+P6+P5+P3"}, {"U6", "P1+P6+P7-P4"}, {"U7", "P1+P6+P7+P5"}};
const Def kResultsABC[] = {{"U1", "P1+P2+bC11"},
                           {"U5", "P1+P6+P5+P3+bC12"},
                           {"U6", "P1+P6+P7-P4+bC21"},
                           {"U7", "P1+P6+P7+P5+bC22"}};
// Intermediate values of the accumulating tables: Table 2 (P5 + beta C22,
// P5 + beta C12, P1 + beta C11, P3 + P5 + beta C12, P4 - beta C21), Tables
// 6-8 (Z1 = C22 - C12, Z2 = C21 - Z1, P7 + beta Z1, P4 - beta Z2, U2 + P7 +
// beta Z1, U4 + beta C12, P2 + beta C11) and Table 9 (Z3 = C12 - C21,
// P5 + beta Z3, P6 + beta C21, W1 = P5 + beta (Z3 + Z1), P3 + P5 + beta Z3,
// U2 + beta C21, U3 + beta C21).
const Def kExtraABC[] = {
    {"C11", "C11"}, {"C12", "C12"}, {"C21", "C21"}, {"C22", "C22"},
    {"Z1", "C22-C12"}, {"Z2", "C21-C22+C12"}, {"Z3", "C12-C21"},
    {nullptr, "P5+bC22"}, {nullptr, "P5+bC12"}, {nullptr, "P1+bC11"}, {nullptr, "P3+P5+bC12"},
    {nullptr, "P4-bC21"}, {nullptr, "P7+bC22-bC12"}, {nullptr, "P4-bC21+bC22-bC12"},
    {nullptr, "P1+P6+P7+bC22-bC12"}, {nullptr, "P1+P6+P5+bC12"}, {nullptr, "P2+bC11"},
    {nullptr, "P5+bC12-bC21"}, {nullptr, "P6+bC21"}, {nullptr, "P5+bC22-bC21"},
    {nullptr, "P3+P5+bC12-bC21"}, {nullptr, "P1+P6+bC21"}, {nullptr, "P1+P6+P7+bC21"},
};

int find(const Graph &g, const char *name) {
  for (size_t i = 0; i < g.nodes.size(); ++i)
    if (g.nodes[i].name == name) return (int)i;
  return -1;
}

void push(Graph &g, const char *name, const char *expr) {
  Node n;
  n.name = name ? name : expr;
  parse(expr, &n.vec);
  g.nodes.push_back(n);
}

// value sets are bit masks of one 64-bit word; location contents are int8
static_assert(sizeof(kAB) / sizeof(Def) + sizeof(kExtraABC) / sizeof(Def) + 4 <= kMaxNodes,
              "candidate values must fit a 64-bit mask");

Graph build_graph(int accumulate) {
  Graph g;
  g.accumulate = accumulate;
  for (const Def &d : kAB) push(g, d.name, d.expr);
  if (accumulate)
    for (const Def &d : kExtraABC) push(g, d.name, d.expr);
  for (const Def &d : accumulate ? kResultsABC : kResultsAB) push(g, d.name, d.expr);

  static const char *in_names[12] = {"A11", "A12", "A21", "A22", "B11", "B12",
                                     "B21", "B22", "C11", "C12", "C21", "C22"};
  for (int l = 0; l < (accumulate ? 12 : 8); ++l) {
    const int i = find(g, in_names[l]);
    g.nodes[i].input = true;
    g.nodes[i].home = l;
    g.inputs |= 1ull << i;
  }
  static const char *res[4] = {"U1", "U5", "U6", "U7"};
  for (int q = 0; q < 4; ++q) {
    const int i = find(g, res[q]);
    g.nodes[i].result = true;
    g.nodes[i].home = SWMM_LOC_C11 + q;
    g.results |= 1ull << i;
  }
  static const char *pa[7] = {"A11", "A12", "S4", "A22", "S1", "S2", "S3"};
  static const char *pb[7] = {"B11", "B21", "B22", "T4", "T1", "T2", "T3"};
  for (int p = 0; p < 7; ++p) g.prod_a[p] = find(g, pa[p]), g.prod_b[p] = find(g, pb[p]);

  // every way of computing each candidate from others
  const int N = (int)g.nodes.size();
  const int ncoef = accumulate ? 4 : 2;
  std::vector<Vec> Pv(7);
  for (int p = 0; p < 7; ++p) {
    Pv[p].sp = SP_C;
    Pv[p].u[p] = 1;
  }
  for (int w = 0; w < N; ++w) {
    Node &W = g.nodes[w];
    if (W.input) continue;
    if (W.vec.sp == SP_C) {
      for (int p = 0; p < 7; ++p) {
        if (W.vec == Pv[p]) W.der.push_back({D_MUL, -1, -1, SWMM_COEF_ONE, (int8_t)p, 1, 0});
        for (int sign = 1; sign >= -1; sign -= 2) {
          Vec sp;
          scaled(Pv[p], sign > 0 ? SWMM_COEF_ONE : SWMM_COEF_NEG, &sp);
          for (int v = 0; v < N; ++v) {
            if (v == w || g.nodes[v].vec.sp != SP_C) continue;
            for (int c = 0; c < ncoef; ++c) {
              Vec cv;
              if (!scaled(g.nodes[v].vec, c, &cv)) continue;
              if (add(sp, cv) == W.vec) W.der.push_back({D_ACC, -1, (int8_t)v, (int8_t)c, (int8_t)p, (int8_t)sign, 0});
            }
          }
        }
      }
    }
    for (int u = 0; u < N; ++u) {
      if (u == w || g.nodes[u].vec.sp != W.vec.sp) continue;
      for (int v = 0; v < N; ++v) {
        if (v == w || v == u || g.nodes[v].vec.sp != W.vec.sp) continue;
        for (int c = 0; c < ncoef; ++c) {
          if (c == SWMM_COEF_ONE && v < u) continue;  // u + v once
          Vec cv;
          if (!scaled(g.nodes[v].vec, c, &cv)) continue;
          if (add(g.nodes[u].vec, cv) == W.vec) W.der.push_back({D_ADD, (int8_t)u, (int8_t)v, (int8_t)c, -1, 1, 0});
        }
      }
    }
    for (Deriv &d : W.der) {
      if (d.type == D_ACC) W.finishers |= 1u << d.prod;
      if (d.type == D_ADD) d.rd = (1ull << d.u) | (1ull << d.v);
      else d.rd = (1ull << g.prod_a[d.prod]) | (1ull << g.prod_b[d.prod]) | (d.type == D_ACC ? 1ull << d.v : 0);
      W.need_any |= d.rd;
    }
  }
  return g;
}

const Graph &graph(int accumulate) {
  static const Graph g0 = build_graph(0), g1 = build_graph(1);
  return accumulate ? g1 : g0;
}

// --------------------------------------------------------------- contracts
struct Contract {
  int kind;    // schedule code, or SWMM_SEARCH_SELF
  bool acc;    // accumulates into the destination
  int clob;    // bit 0: overwrites the left operand, bit 1: the right one
};
// Tables 1-9 and the Section 5.1 variant of Table 4 (whose partial
// overwrites, like Table 8's, count as overwriting the whole operand here)
const Contract kContracts[] = {
    {SWMM_T1_DHSS, false, 0}, {SWMM_T2_HLJJTT, true, 0}, {SWMM_T3_IP, false, 3},
    {SWMM_T4_OVL, false, 1},  {SWMM_T5_OVR, false, 2},   {SWMM_T6_ACLR, true, 3},
    {SWMM_T7_ACCR, true, 2},  {SWMM_T8_ACR, true, 2},    {SWMM_T9_ACC, true, 0},
    {SWMM_T4M_OVL, false, 1},
};

// Block shapes (Section 5.3).  With relative operand sizes m x k (A), k x n
// (B) and m x n (C), the blocks of A, B and C are halved alike, a value of
// A, B or C has its matrix's block shape, and a value fits a block when
// neither dimension is larger.  Temporaries hold any value.  Tables 4-7 and
// 9 need m = k = n; Table 3 needs k = n <= m.
struct Dims {
  int m = 1, k = 1, n = 1;
  bool square() const { return m == k && k == n; }
};
Dims dims_of(const swmm_search_spec &s) {
  Dims d;
  if (s.m > 0 && s.k > 0 && s.n > 0) d.m = s.m, d.k = s.k, d.n = s.n;
  return d;
}
bool fits(const Dims &d, int space, int loc) {
  if (loc >= SWMM_LOC_X) return true;
  const int vr = space == SP_B ? d.k : d.m, vc = space == SP_A ? d.k : d.n;
  const int lr = loc >= SWMM_LOC_B11 && loc < SWMM_LOC_C11 ? d.k : d.m;
  const int lc = loc < SWMM_LOC_B11 ? d.k : d.n;
  return vr <= lr && vc <= lc;
}
bool kind_allowed(const Dims &d, int kind) {
  if (d.square() || kind == SWMM_SEARCH_SELF) return true;
  switch (kind) {
    case SWMM_T1_DHSS: case SWMM_T2_HLJJTT: case SWMM_T8_ACR: return true;
    case SWMM_T3_IP: return d.k == d.n && d.n <= d.m;
    default: return false;  // the square-only tables
  }
}

// The schedule searched for overwrites an operand of its own recursive calls
// where its spec lets it overwrite a block of that matrix.
int self_clobber(const swmm_search_spec &s) {
  return ((s.preserve & 0x0f) != 0x0f ? 1 : 0) | ((s.preserve & 0xf0) != 0xf0 ? 2 : 0);
}

// ------------------------------------------------------------------ search
constexpr int8_t kEmpty = -1;

struct State {
  int8_t loc[SWMM_NLOC];
  uint64_t done;     // values computed so far (inputs count as computed)
  uint8_t prod;      // products used
  uint8_t written;   // blocks of A and B written or overwritten
  uint8_t copies;
};

inline uint64_t mix(uint64_t x) {  // splitmix64 finaliser
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Open-addressing set of 128-bit state fingerprints, each with the rows and
// block additions of the path it was last expanded on.  A state reached
// again is expanded again unless that path had no more rows and no more
// additions (then every continuation was already tried within the limits).
// The table starts small and doubles up to the state limit; it never holds
// more than the limit's number of states.
class Visited {
 public:
  bool init(int64_t max_states) {
    size_ = 0;
    limit_ = (uint64_t)std::max<int64_t>(max_states, 1);
    max_cap_ = 1;
    while (max_cap_ < 2 * (uint64_t)max_states) max_cap_ <<= 1;
    return alloc(std::min<uint64_t>(max_cap_, 1u << 16));
  }
  // Slot for a fingerprint, or -1 when nothing is to be done (dominated, or
  // *full: the state limit is reached).
  int64_t probe(uint64_t h1, uint64_t h2, int depth, int adds, bool *full) {
    h1 |= 1;
    if (size_ * 2 >= cap_ && cap_ < max_cap_ && !grow()) {
      *full = true;
      return -1;
    }
    for (uint64_t i = h1 & (cap_ - 1);; i = (i + 1) & (cap_ - 1)) {
      const Slot &s = tab_[i];
      if (s.h1 == 0) {
        if (size_ * 2 >= cap_ || size_ >= limit_) {
          *full = true;
          return -1;
        }
        return (int64_t)i;
      }
      if (s.h1 == h1 && s.h2 == h2) return (depth < s.depth || adds < s.adds) ? (int64_t)i : -1;
    }
  }
  void insert(int64_t i, uint64_t h1, uint64_t h2, int depth, int adds) {
    Slot &s = tab_[i];
    if (s.h1 == 0) ++size_;
    s.h1 = h1 | 1;
    s.h2 = h2;
    s.depth = (uint8_t)depth;
    s.adds = (uint8_t)adds;
  }
  int64_t size() const { return (int64_t)size_; }

 private:
  struct Slot {
    uint64_t h1, h2;
    uint8_t depth, adds;
  };
  bool alloc(uint64_t cap) {
    std::vector<Slot> t;
    try {
      t.assign(cap, Slot{0, 0, 0, 0});
    } catch (...) {
      return false;
    }
    tab_.swap(t);
    cap_ = cap;
    return true;
  }
  bool grow() {
    std::vector<Slot> old;
    old.swap(tab_);
    if (!alloc(cap_ * 2)) {
      tab_.swap(old);
      return false;
    }
    for (const Slot &s : old) {
      if (s.h1 == 0) continue;
      uint64_t i = s.h1 & (cap_ - 1);
      while (tab_[i].h1 != 0) i = (i + 1) & (cap_ - 1);
      tab_[i] = s;
    }
    return true;
  }
  std::vector<Slot> tab_;
  uint64_t cap_ = 0, max_cap_ = 0, size_ = 0, limit_ = 1;
};

class Search {
 public:
  Search(const swmm_search_spec &s, const Graph &g) : sp_(s), g_(g) {
    nloc_ = 12 + s.temps;
    N_ = (int)g.nodes.size();
    for (int b = 0; b < 8; ++b)
      if (s.preserve >> b & 1) preserved_ |= 1ull << home_of(b);
    dims_ = dims_of(s);
    for (const Contract &c : kContracts)
      if ((s.kinds >> c.kind & 1) && kind_allowed(dims_, c.kind)) con_.push_back(c);
    if (s.kinds >> SWMM_SEARCH_SELF & 1) con_.push_back({SWMM_SEARCH_SELF, s.accumulate != 0, self_clobber(s)});
    all_clob_ = 3;
    for (const Contract &c : con_) all_clob_ &= c.clob;
    // memory-frugal contracts (more overwriting) first
    std::stable_sort(con_.begin(), con_.end(), [](const Contract &a, const Contract &b) {
      return __builtin_popcount(a.clob) > __builtin_popcount(b.clob);
    });
  }

  // One depth-first search within `cap` states; with the portfolio order,
  // searches in both orders with budgets growing fourfold, until one finds
  // a schedule or visits every state (a proof), or the states run out.
  bool run(swmm_search_result *res, std::vector<swmm_search_row> *out) {
    const int64_t cap = sp_.max_states > 0 ? sp_.max_states : (int64_t)1 << 26;
    int64_t used = 0;
    bool done = false;
    for (int round = 0; !done; ++round) {
      int64_t budget = cap - used;
      if (sp_.order == SWMM_ORDER_PORTFOLIO) budget = std::min<int64_t>(budget, (int64_t)1 << (16 + 2 * (round / 2)));
      descending_ = sp_.order == SWMM_ORDER_DESCENDING || (sp_.order == SWMM_ORDER_PORTFOLIO && round % 2 == 1);
      if (!vis_.init(budget)) return false;
      std::fill(dead_.begin(), dead_.end(), 0);
      full_ = false;
      path_.clear();
      State s{};
      for (int l = 0; l < SWMM_NLOC; ++l) s.loc[l] = kEmpty;
      for (int i = 0; i < N_; ++i)
        if (g_.nodes[i].input) s.loc[g_.nodes[i].home] = (int8_t)i;
      s.done = g_.inputs;
      const uint64_t want = normalize(&s);
      found_ = dfs(s, 0, 0, want);
      used += vis_.size();
      done = found_ || !full_ || used >= cap || sp_.order != SWMM_ORDER_PORTFOLIO;
    }
    res->found = found_ ? 1 : 0;
    res->exhausted = (!found_ && !full_) ? 1 : 0;
    res->states = used;
    if (found_) *out = best_;
    return true;
  }

 private:
  int home_of(int l) const {
    for (int i = 0; i < N_; ++i)
      if (g_.nodes[i].input && g_.nodes[i].home == l) return i;
    return -1;
  }
  uint64_t present(const State &s) const {
    uint64_t m = 0;
    for (int l = 0; l < nloc_; ++l)
      if (s.loc[l] != kEmpty) m |= 1ull << s.loc[l];
    return m;
  }
  bool at_home(const State &s, int i) const { return s.loc[g_.nodes[i].home] == i; }
  bool goal(const State &s) const {
    for (uint64_t m = g_.results | preserved_; m; m &= m - 1)
      if (!at_home(s, __builtin_ctzll(m))) return false;
    return true;
  }
  // a product is used once; without `recompute` a value is computed once
  bool can_compute(const State &s, const Deriv &d, int w) const {
    if (sp_.exclude >> w & 1) return false;
    if (d.type == D_ADD) return !(s.done >> w & 1) || (sp_.recompute && g_.nodes[w].vec.sp != SP_C);
    return !(s.prod >> d.prod & 1);
  }
  // A value must be produced when it is a result or a preserved block not
  // in its place, or is absent and wanted; the values its remaining
  // derivations read are wanted.  Everything else a block holds is dead.
  bool to_produce(const State &s, uint64_t pres, int w) const {
    const Node &n = g_.nodes[w];
    if ((n.result || (preserved_ >> w & 1)) && !at_home(s, w)) return true;
    return !(pres >> w & 1);
  }
  uint64_t wanted(const State &s, uint64_t pres) const {
    uint64_t want = g_.results | preserved_, seen = 0;
    for (uint64_t todo = want; todo;) {
      const int w = __builtin_ctzll(todo);
      todo &= todo - 1;
      seen |= 1ull << w;
      // a present value is expanded too when it may be formed again later
      // (an operand sum under `recompute`): what it is formed from stays
      if (g_.nodes[w].input ||
          (!to_produce(s, pres, w) && !(sp_.recompute && g_.nodes[w].vec.sp != SP_C)))
        continue;
      for (const Deriv &d : g_.nodes[w].der) {
        if (!can_compute(s, d, w)) continue;
        const uint64_t r = d.rd;
        want |= r;
        todo |= r & ~seen;
      }
    }
    return want;
  }
  // clear blocks holding dead values (they are free pebbles)
  uint64_t normalize(State *s) const {
    const uint64_t want = wanted(*s, present(*s));
    for (int l = 0; l < nloc_; ++l)
      if (s->loc[l] != kEmpty && !(want >> s->loc[l] & 1)) s->loc[l] = kEmpty;
    return want;
  }
  // results still obtainable (over-approximation: products may be shared
  // between values here), preserved blocks still restorable
  bool feasible(const State &s, uint64_t pres, uint64_t want) const {
    uint64_t obt = pres;
    for (bool changed = true; changed;) {
      changed = false;
      for (uint64_t m = want & ~obt; m; m &= m - 1) {
        const int w = __builtin_ctzll(m);
        for (const Deriv &d : g_.nodes[w].der) {
          if (!can_compute(s, d, w)) continue;
          if ((d.rd & ~obt) == 0) {
            obt |= 1ull << w;
            changed = true;
            break;
          }
        }
      }
    }
    if ((g_.results & ~obt) != 0) return false;
    const bool can_copy = s.copies < sp_.max_copies;
    for (uint64_t m = preserved_; m; m &= m - 1) {
      const int i = __builtin_ctzll(m);
      if (at_home(s, i)) continue;
      if (!(pres >> i & 1) || !can_copy) return false;
    }
    return true;
  }
  // Blocks of A and B already overwritten that need not be restored are
  // interchangeable with the temporaries: their contents are sorted as one
  // group.  What is left of `done` that matters: absent wanted values.
  void fingerprint(const State &s, uint64_t pres, uint64_t want, uint64_t *h1, uint64_t *h2) const {
    int8_t grp[16];
    int ng = 0;
    uint64_t w[3] = {0, 0, 0};
    int bit = 0;
    for (int l = 0; l < nloc_; ++l) {
        if (scratch(s, l)) {
        grp[ng++] = s.loc[l];
      } else {
        w[bit / 64] |= (uint64_t)(uint8_t)s.loc[l] << (bit % 64);
        bit += 8;
        if (bit % 64 == 0 && bit / 64 > 2) break;
      }
    }
    std::sort(grp, grp + ng);
    uint64_t gw[2] = {0, 0};
    for (int k = 0; k < ng; ++k) gw[k / 8] |= (uint64_t)(uint8_t)grp[k] << (8 * (k % 8));
    const uint64_t meta = (uint64_t)s.prod | (uint64_t)s.written << 8 | (uint64_t)s.copies << 16;
    const uint64_t dn = s.done & want & ~pres;
    uint64_t a = mix(meta ^ 0x243f6a8885a308d3ull), b = mix(meta + 0x13198a2e03707344ull);
    for (uint64_t x : {w[0], w[1], w[2], gw[0], gw[1], dn}) {
      a = mix(a ^ x);
      b = mix(b + 0x9e3779b97f4a7c15ull * (x ^ 0xa4093822299f31d0ull));
    }
    *h1 = a;
    *h2 = b;
  }
  void wrote(State &s, int l) const {
    if (l < 8) s.written |= (uint8_t)(1u << l);
  }
  int first_loc(const State &s, int node, int avoid = -1) const {
    for (int l = 0; l < nloc_; ++l)
      if (s.loc[l] == node && l != avoid) return l;
    return -1;
  }

  // Lower bound on the blocks of A and B written by the end: an input block
  // still at home that a pending product reads through calls that all
  // overwrite that operand will be written, unless a copy of it is made
  // first (each remaining copy spares at most one such block).
  int written_bound(const State &s) const {
    uint32_t w = s.written;
    for (int p = 0; p < 7; ++p) {
      if (s.prod >> p & 1) continue;
      for (int side = 0; side < 2; ++side) {
        const int x = side ? g_.prod_b[p] : g_.prod_a[p];
        if (!g_.nodes[x].input || !(all_clob_ >> side & 1)) continue;
        const int l = g_.nodes[x].home;
        if (s.loc[l] == x && first_loc(s, x, l) < 0) w |= 1u << l;
      }
    }
    const int spare = std::min(sp_.max_copies - s.copies, __builtin_popcount(w & ~s.written));
    return __builtin_popcount(w) - spare;
  }
  // Lower bound on the rows still to come: one per pending product, one per
  // absent operand sum of a pending product, one per result not in place
  // beyond those a product row can leave in place.
  int rows_bound(const State &s, uint64_t pres) const {
    const int unused = 7 - __builtin_popcount(s.prod);
    return unused + absent_operands(s, pres) + unfinished(s);
  }
  // absent operand sums of pending products (each needs an addition)
  int absent_operands(const State &s, uint64_t pres) const {
    uint64_t ops = 0;
    for (int p = 0; p < 7; ++p)
      if (!(s.prod >> p & 1)) ops |= (1ull << g_.prod_a[p]) | (1ull << g_.prod_b[p]);
    return __builtin_popcount(ops & ~pres & ~g_.inputs);
  }
  // Results not in place that no pending product can finish: a result's
  // last row is an addition unless it accumulates a product into the rest
  // of the result, and each product finishes at most one result (a
  // bipartite matching of pending results to pending products).
  int unfinished(const State &s) const {
    int res[4], n = 0;
    for (uint64_t m = g_.results; m; m &= m - 1) {
      const int r = __builtin_ctzll(m);
      if (!at_home(s, r)) res[n++] = r;
    }
    int owner[7] = {-1, -1, -1, -1, -1, -1, -1};
    int matched = 0;
    for (int i = 0; i < n; ++i) {
      bool seen[7] = {};
      if (augment(s, res, i, owner, seen)) ++matched;
    }
    return n - matched;
  }
  bool augment(const State &s, const int *res, int i, int *owner, bool *seen) const {
    const unsigned fin = g_.nodes[res[i]].finishers & ~s.prod;
    for (int p = 0; p < 7; ++p) {
      if (!(fin >> p & 1) || seen[p]) continue;
      seen[p] = true;
      if (owner[p] < 0 || augment(s, res, owner[p], owner, seen)) {
        owner[p] = i;
        return true;
      }
    }
    return false;
  }

  // Lower bound on the block additions still to come: one per absent
  // operand sum of a pending product, one per result no pending product
  // can finish.
  int adds_bound(const State &s, uint64_t pres) const { return absent_operands(s, pres) + unfinished(s); }

  bool step(State n, int depth, int adds, const swmm_search_row &row) {
    if (sp_.max_written >= 0 && written_bound(n) > sp_.max_written) return false;
    const uint64_t want = normalize(&n);
    path_.push_back(row);
    const bool ok = dfs(n, depth + 1, adds + (row.op == SWMM_ROW_ADD ? 1 : 0), want);
    if (!ok) path_.pop_back();
    return ok;
  }
  // blocks interchangeable with the temporaries (only when all blocks have
  // one shape)
  bool scratch(const State &s, int l) const {
    return l >= 12 || (dims_.square() && l < 8 && (s.written >> l & 1) && !(sp_.preserve >> l & 1));
  }
  // Destinations worth trying: one free block of the scratch group stands
  // for all of them, and a block whose value could not be had again is
  // never written over: a result in place (when values are computed once),
  // a preserved block in place, an operand of a pending product that is
  // an input or cannot be computed again.
  uint32_t dests(const State &s) const {
    uint64_t keep = 0;
    for (uint64_t m = g_.results | preserved_; m; m &= m - 1) {
      const int i = __builtin_ctzll(m);
      if (at_home(s, i)) keep |= 1ull << i;  // results are C values: never formed twice
    }
    for (int p = 0; p < 7; ++p) {
      if (s.prod >> p & 1) continue;
      for (const int x : {g_.prod_a[p], g_.prod_b[p]})
        if (g_.nodes[x].input || !sp_.recompute) keep |= 1ull << x;
    }
    uint32_t m = 0;
    bool free_scratch = false;
    for (int l = 0; l < nloc_; ++l) {
      const int8_t x = s.loc[l];
      if (x == kEmpty) {
        if (scratch(s, l)) {
          if (free_scratch) continue;
          free_scratch = true;
        }
      } else if ((keep >> x & 1) && first_loc(s, x, l) < 0) {
        continue;
      }
      m |= 1u << l;
    }
    return m;
  }

  bool dfs(const State &s, int depth, int adds, uint64_t want) {
    if (sp_.max_adds >= 0 && adds > sp_.max_adds) return false;
    if (goal(s)) {
      best_ = path_;
      return true;
    }
    if (full_) return false;
    const uint64_t pres = present(s);
    if (depth + rows_bound(s, pres) > sp_.max_rows) return false;
    if (sp_.max_adds >= 0 && adds + adds_bound(s, pres) > sp_.max_adds) return false;
    uint64_t h1, h2;
    fingerprint(s, pres, want, &h1, &h2);
    const int cost_adds = sp_.max_adds >= 0 ? adds : 0;  // additions matter only under a limit
    const int64_t slot = vis_.probe(h1, h2, depth, cost_adds, &full_);
    if (slot < 0) return false;
    // dead states go to a lossy cache (an evicted one is only re-checked)
    uint64_t &dead = dead_[h1 & (kDeadSlots - 1)];
    if (dead == (h2 | 1)) return false;
    if (!feasible(s, pres, want)) {
      dead = h2 | 1;
      return false;
    }
    vis_.insert(slot, h1, h2, depth, cost_adds);
    const uint32_t dmask = dests(s);

    for (uint64_t m = want & ~g_.inputs; m;) {
      // values in list order, or (descending) results and sums of products first
      const int w = descending_ ? 63 - __builtin_clzll(m) : __builtin_ctzll(m);
      m &= ~(1ull << w);
      if (!to_produce(s, pres, w)) continue;
      for (const Deriv &d : g_.nodes[w].der) {
        if (!can_compute(s, d, w)) continue;
        if ((d.rd & ~pres) != 0) continue;
        if (d.type == D_ADD) {
          for (int dst = 0; dst < nloc_; ++dst) {
            if (!(dmask >> dst & 1) || s.loc[dst] == w || !fits(dims_, g_.nodes[w].vec.sp, dst)) continue;
            // read an operand from dst when dst holds it (in place)
            const int lu = s.loc[dst] == d.u ? dst : first_loc(s, d.u);
            const int lv = s.loc[dst] == d.v ? dst : first_loc(s, d.v);
            State n = s;
            n.loc[dst] = (int8_t)w;
            n.done |= 1ull << w;
            wrote(n, dst);
            const swmm_search_row r{SWMM_ROW_ADD, dst, lu, lv, d.coef, 0, 1, 0, w};
            if (step(n, depth, adds, r)) return true;
            if (full_) return false;
          }
          continue;
        }
        const int a = g_.prod_a[d.prod], b = g_.prod_b[d.prod];
        for (const Contract &c : con_) {
          if (c.acc != (d.type == D_ACC)) continue;
          for (int dst = 0; dst < nloc_; ++dst) {
            if (!(dmask >> dst & 1) || !fits(dims_, SP_C, dst)) continue;
            if (d.type == D_ACC && s.loc[dst] != d.v) continue;
            // operand copies: branch over the copies a call overwrites
            for (int la = 0; la < nloc_; ++la) {
              if (s.loc[la] != a || la == dst) continue;
              if (!(c.clob & 1) && la != first_loc(s, a, dst)) continue;
              for (int lb = 0; lb < nloc_; ++lb) {
                if (s.loc[lb] != b || lb == dst) continue;
                if (!(c.clob & 2) && lb != first_loc(s, b, dst)) continue;
                State n = s;
                n.loc[dst] = (int8_t)w;
                n.done |= 1ull << w;
                n.prod |= (uint8_t)(1u << d.prod);
                wrote(n, dst);
                if (c.clob & 1) n.loc[la] = kEmpty, wrote(n, la);
                if (c.clob & 2) n.loc[lb] = kEmpty, wrote(n, lb);
                const swmm_search_row r{SWMM_ROW_MUL, dst, la, lb, d.coef, d.type == D_ACC ? 1 : 0, d.sign, c.kind, w};
                if (step(n, depth, adds, r)) return true;
                if (full_) return false;
              }
            }
          }
        }
      }
    }
    if (s.copies < sp_.max_copies) {
      for (uint64_t m = pres; m; m &= m - 1) {
        const int x = __builtin_ctzll(m);
        const int from = first_loc(s, x);
        for (int dst = 0; dst < nloc_; ++dst) {
          const int held = s.loc[dst];
          if (!(dmask >> dst & 1) || held == x || !fits(dims_, g_.nodes[x].vec.sp, dst)) continue;
          if (held != kEmpty) continue;  // into a free block
          State n = s;
          n.loc[dst] = (int8_t)x;
          n.copies++;
          wrote(n, dst);
          const swmm_search_row r{SWMM_ROW_COPY, dst, from, -1, 0, 0, 1, 0, x};
          if (step(n, depth, adds, r)) return true;
          if (full_) return false;
        }
      }
    }
    return false;
  }

  static constexpr uint64_t kDeadSlots = 1u << 20;
  std::vector<uint64_t> dead_ = std::vector<uint64_t>(kDeadSlots, 0);
  const swmm_search_spec &sp_;
  const Graph &g_;
  int N_ = 0, nloc_ = 12;
  uint64_t preserved_ = 0;
  Dims dims_;
  int all_clob_ = 0;  // operands every allowed call overwrites (bit 0 left, 1 right)
  std::vector<Contract> con_;
  Visited vis_;
  std::vector<swmm_search_row> path_, best_;
  bool found_ = false, full_ = false, descending_ = false;
};

// ------------------------------------------------------------------ replay
// Plays the rows of a given schedule under the same rules; returns the
// index of the first row that is not a legal move (nrows when all are).
int replay(const swmm_search_spec &sp, const Graph &g, swmm_search_row *rows, int nrows, bool *goal,
           uint32_t *written, uint32_t *temps) {
  const int nloc = 12 + sp.temps;
  const Dims dm = dims_of(sp);
  int8_t loc[SWMM_NLOC];
  for (int l = 0; l < SWMM_NLOC; ++l) loc[l] = kEmpty;
  for (size_t i = 0; i < g.nodes.size(); ++i)
    if (g.nodes[i].input) loc[g.nodes[i].home] = (int8_t)i;
  uint64_t done = g.inputs;
  uint32_t prod = 0;
  int copies = 0;
  *written = *temps = 0;
  *goal = false;
  auto node_of = [&](const Vec &v) {
    for (size_t i = 0; i < g.nodes.size(); ++i)
      if (g.nodes[i].vec == v) return (int)i;
    return -1;
  };
  auto mark = [&](int l) {
    if (l < 8) *written |= 1u << l;
    if (l >= 12) *temps |= 1u << (l - 12);
  };
  for (int i = 0; i < nrows; ++i) {
    swmm_search_row &r = rows[i];
    if (r.dst < 0 || r.dst >= nloc) return i;
    const bool s1ok = r.s1 >= 0 && r.s1 < nloc && loc[r.s1] != kEmpty;
    if (!s1ok) return i;
    if (r.op == SWMM_ROW_COPY) {
      if (r.dst == r.s1 || copies >= sp.max_copies || !fits(dm, g.nodes[loc[r.s1]].vec.sp, r.dst)) return i;
      ++copies;
      loc[r.dst] = loc[r.s1];
      r.node = loc[r.s1];
      mark(r.dst);
      continue;
    }
    if (r.s2 < 0 || r.s2 >= nloc || loc[r.s2] == kEmpty || r.s2 == r.s1) return i;
    if (r.coef < 0 || r.coef > 3 || (!sp.accumulate && r.coef > 1)) return i;
    if (r.op == SWMM_ROW_ADD) {
      const Vec &u = g.nodes[loc[r.s1]].vec, &v = g.nodes[loc[r.s2]].vec;
      Vec cv;
      if (u.sp != v.sp || !scaled(v, r.coef, &cv)) return i;
      const int w = node_of(add(u, cv));
      if (w < 0 || g.nodes[w].input || ((done >> w & 1) && !(sp.recompute && g.nodes[w].vec.sp != SP_C))) return i;
      if (!fits(dm, u.sp, r.dst)) return i;
      loc[r.dst] = (int8_t)w;
      done |= 1ull << w;
      r.node = w;
      mark(r.dst);
      continue;
    }
    if (r.op != SWMM_ROW_MUL || r.dst == r.s1 || r.dst == r.s2 || (r.sign != 1 && r.sign != -1)) return i;
    int p = -1;
    for (int q = 0; q < 7; ++q)
      if (g.prod_a[q] == loc[r.s1] && g.prod_b[q] == loc[r.s2]) p = q;
    if (p < 0 || (prod >> p & 1)) return i;
    Contract c{-1, false, 0};
    if (r.kind >= 0 && r.kind <= 31 && (sp.kinds >> r.kind & 1)) {
      if (r.kind == SWMM_SEARCH_SELF) c = {SWMM_SEARCH_SELF, sp.accumulate != 0, self_clobber(sp)};
      for (const Contract &k : kContracts)
        if (k.kind == r.kind) c = k;
    }
    if (c.kind < 0 || c.acc != (r.accumulate != 0) || !kind_allowed(dm, c.kind) || !fits(dm, SP_C, r.dst)) return i;
    Vec pv;
    pv.sp = SP_C;
    pv.u[p] = (int8_t)r.sign;
    if (r.accumulate) {
      if (loc[r.dst] == kEmpty) return i;
      Vec cv;
      if (!scaled(g.nodes[loc[r.dst]].vec, r.coef, &cv)) return i;
      pv = add(pv, cv);
    } else if (r.sign != 1) {
      return i;
    }
    const int w = node_of(pv);
    if (w < 0 || g.nodes[w].input) return i;
    loc[r.dst] = (int8_t)w;
    done |= 1ull << w;
    prod |= 1u << p;
    r.node = w;
    mark(r.dst);
    if (c.clob & 1) loc[r.s1] = kEmpty, mark(r.s1);
    if (c.clob & 2) loc[r.s2] = kEmpty, mark(r.s2);
  }
  bool ok = true;
  for (size_t i = 0; i < g.nodes.size(); ++i) {
    const Node &n = g.nodes[i];
    const bool keep = n.result || (n.input && n.home < 8 && (sp.preserve >> n.home & 1));
    if (keep && loc[n.home] != (int)i) ok = false;
  }
  *goal = ok;
  return nrows;
}

bool spec_ok(const swmm_search_spec *spec) {
  if (!spec || (spec->accumulate != 0 && spec->accumulate != 1)) return false;
  if (spec->temps < 0 || spec->temps > 3 || spec->max_copies < 0 || spec->max_rows < 1 ||
      spec->max_rows > SWMM_SEARCH_MAX_ROWS || (spec->preserve & ~0xffu) || spec->max_adds > 255 ||
      spec->m < 0 || spec->k < 0 || spec->n < 0)
    return false;
  const uint32_t known = (1u << SWMM_T1_DHSS) | (1u << SWMM_T2_HLJJTT) | (1u << SWMM_T3_IP) | (1u << SWMM_T4_OVL) |
                         (1u << SWMM_T5_OVR) | (1u << SWMM_T6_ACLR) | (1u << SWMM_T7_ACCR) | (1u << SWMM_T8_ACR) |
                         (1u << SWMM_T9_ACC) | (1u << SWMM_T4M_OVL) | (1u << SWMM_SEARCH_SELF);
  if (spec->order < SWMM_ORDER_ASCENDING || spec->order > SWMM_ORDER_PORTFOLIO) return false;
  return (spec->kinds & ~known) == 0;
}

}  // namespace

namespace swmm {
namespace {

// schedule codes of swmm.h <-> kinds of the executor
constexpr int kCodeOfKind[NKIND] = {SWMM_T1_DHSS, SWMM_T2_HLJJTT, SWMM_T3_IP,   SWMM_T4_OVL,  SWMM_T4M_OVL,
                                    SWMM_T5_OVR,  SWMM_T6_ACLR,   SWMM_T7_ACCR, SWMM_T8_ACR, SWMM_T9_ACC};
static_assert(K_T1 == 0 && K_OVLM == 4 && K_ACC == 9, "kind order");
Kind kind_of_code(int c) {
  for (int k = 0; k < NKIND; ++k)
    if (kCodeOfKind[k] == c) return (Kind)k;
  return K_CUSTOM;
}

}  // namespace

bool lower_schedule(const swmm_search_spec &spec, const swmm_search_row *rows, int nrows, CustomSchedule *out,
                    std::string *err) {
  if (!spec_ok(&spec) || nrows < 1 || nrows > SWMM_SEARCH_MAX_ROWS || !rows) {
    *err = "bad schedule spec or row count";
    return false;
  }
  const Graph &g = graph(spec.accumulate);
  std::vector<swmm_search_row> r(rows, rows + nrows);
  bool goal;
  uint32_t w, t;
  const int legal = replay(spec, g, r.data(), nrows, &goal, &w, &t);
  if (legal < nrows) {
    *err = "row " + std::to_string(legal + 1) + " is not a legal move";
    return false;
  }
  if (!goal) {
    *err = "the results or the preserved blocks do not end in place";
    return false;
  }
  static const Coef cf[4] = {CF_ONE, CF_NEG, CF_BETA, CF_NBETA};
  out->rows.clear();
  for (const swmm_search_row &x : r) {
    Row y{};
    y.dst = (Loc)x.dst;
    y.s1 = (Loc)x.s1;
    y.s2 = x.op == SWMM_ROW_COPY ? (Loc)x.s1 : (Loc)x.s2;
    y.shape = (Shape)g.nodes[x.node].vec.sp;  // SP_A, SP_B, SP_C match SH_A, SH_B, SH_C
    if (x.op == SWMM_ROW_ADD) {
      y.op = OP_ADD;
      y.c1 = CF_ONE;
      y.c2 = cf[x.coef];
    } else if (x.op == SWMM_ROW_COPY) {
      y.op = OP_COPY;
    } else {
      y.op = OP_MUL;
      y.shape = SH_C;
      y.c1 = x.sign > 0 ? CF_ALPHA : CF_NALPHA;
      y.kind = kind_of_code(x.kind);
      y.acc = x.accumulate != 0;
      y.cacc = y.acc ? cf[x.coef] : CF_ONE;
    }
    out->rows.push_back(y);
  }
  out->accumulate = spec.accumulate != 0;
  out->preserve = spec.preserve;
  out->temps = __builtin_popcount(t);
  return true;
}

}  // namespace swmm

extern "C" {

int swmm_schedule_search(const swmm_search_spec *spec, swmm_search_row *rows, int32_t max_rows_out,
                         swmm_search_result *res) {
  if (!spec_ok(spec) || !res || (!rows && max_rows_out > 0) || max_rows_out < 0) return SWMM_EINVAL;
  memset(res, 0, sizeof(*res));
  const Graph &g = graph(spec->accumulate);
  Search s(*spec, g);
  std::vector<swmm_search_row> out;
  if (!s.run(res, &out)) return SWMM_ENOMEM;
  if (res->found) {
    bool goal;
    uint32_t w, t;
    replay(*spec, g, out.data(), (int)out.size(), &goal, &w, &t);
    res->written = __builtin_popcount(w);
    res->temps_used = __builtin_popcount(t);
    res->nrows = (int32_t)std::min<size_t>(out.size(), (size_t)max_rows_out);
    for (int i = 0; i < res->nrows; ++i) rows[i] = out[i];
  }
  return SWMM_OK;
}

int swmm_schedule_check(const swmm_search_spec *spec, swmm_search_row *rows, int32_t nrows,
                        swmm_search_result *res) {
  if (!spec_ok(spec) || !res || nrows < 0 || (!rows && nrows > 0)) return SWMM_EINVAL;
  memset(res, 0, sizeof(*res));
  bool goal;
  uint32_t w, t;
  res->nrows = replay(*spec, graph(spec->accumulate), rows, nrows, &goal, &w, &t);
  res->found = (res->nrows == nrows && goal) ? 1 : 0;
  res->written = __builtin_popcount(w);
  res->temps_used = __builtin_popcount(t);
  return SWMM_OK;
}

int swmm_table_rows(int32_t sched, swmm_search_row *rows, int32_t max_rows, int32_t *nrows) {
  using namespace swmm;
  const Kind k = kind_of_code(sched);
  if (k == K_CUSTOM || !nrows || max_rows < 0 || (!rows && max_rows > 0)) return SWMM_EINVAL;
  const std::vector<Row> &t = *kind_info(k).table;
  *nrows = (int32_t)t.size();
  if ((int)t.size() > max_rows) return SWMM_EINVAL;
  auto coef_of = [](Coef c) {
    switch (c) {
      case CF_NEG: return SWMM_COEF_NEG;
      case CF_BETA: return SWMM_COEF_BETA;
      case CF_NBETA: return SWMM_COEF_NBETA;
      default: return SWMM_COEF_ONE;
    }
  };
  for (size_t i = 0; i < t.size(); ++i) {
    const Row &y = t[i];
    swmm_search_row &x = rows[i];
    x = swmm_search_row{};
    x.dst = y.dst;
    x.s1 = y.s1;
    x.s2 = y.s2;
    x.sign = 1;
    x.node = -1;
    if (y.op == OP_ADD) {
      x.op = SWMM_ROW_ADD;
      // rows are u + c v; a leading -1 puts the other operand first
      if (y.c1 == CF_ONE) {
        x.coef = coef_of(y.c2);
      } else {
        x.s1 = y.s2;
        x.s2 = y.s1;
        x.coef = coef_of(y.c1);
        if (y.c2 != CF_ONE) return SWMM_EUNSUPPORTED;
      }
    } else if (y.op == OP_COPY) {
      x.op = SWMM_ROW_COPY;
      x.s2 = -1;
    } else {
      x.op = SWMM_ROW_MUL;
      x.sign = y.c1 == CF_NALPHA ? -1 : 1;
      x.kind = kCodeOfKind[y.kind];
      x.accumulate = y.acc ? 1 : 0;
      x.coef = y.acc ? coef_of(y.cacc) : SWMM_COEF_ONE;
    }
  }
  return SWMM_OK;
}

const char *swmm_search_node_name(int32_t accumulate, int32_t node) {
  if (accumulate != 0 && accumulate != 1) return nullptr;
  const Graph &g = graph(accumulate);
  if (node < 0 || node >= (int)g.nodes.size()) return nullptr;
  return g.nodes[node].name.c_str();
}

int32_t swmm_search_node_count(int32_t accumulate) {
  if (accumulate != 0 && accumulate != 1) return 0;
  return (int32_t)graph(accumulate).nodes.size();
}

}  // extern "C"
