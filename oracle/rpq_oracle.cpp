// CPU oracle for regular path queries (RPQ) and conjunctive RPQs (CRPQ).
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
// load this file; only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference legs use it. It shares no code with the CUDA path.
//
// What it computes is the plain definition of the paper's problem:
//   * RPQ (Definition 1, Section 2.1): the set of pairs (x, y) such that some
//     directed path from x to y spells a word of L(rho).  Evaluated the
//     automata way (Section 2.2, "Automata-based approach"): for every start
//     vertex, a breadth-first search over product vertices
//     (data vertex, automaton state) with a per-start visited set (one flag
//     per product vertex), adding
//     (start, v) whenever an accepting state is reached.  The automaton is a
//     Thompson epsilon-NFA with explicit epsilon-closures, so no DFA is
//     involved in the result.  There is no hop limit: the search runs until
//     the queue is empty (cf. Section 3, Challenge 1).
//   * CRPQ (Definition 2, Section 2.1): all maps f from query variables to
//     data vertices with (1) equal vertex labels where the variable has one
//     and (2) every atom x -rho-> y satisfied by (f(x), f(y)).  Evaluated by
//     nested loops over the variables in declaration order.
//   * Work counter W: the number of product-edge relaxations a product-graph
//     traversal over the MINIMAL (trimmed, partial) DFA performs, i.e. the sum
//     over start vertices s, product vertices (v, q) reachable from (s, q0),
//     and labels l with a transition out of q, of deg_l(v).  The minimal DFA
//     is unique for a language, so W does not depend on how a DFA is built.
//     This file builds it by subset construction from its own Thompson NFA
//     followed by Moore partition refinement.
//
// Readings of the paper taken here (each also listed in the design notes):
//   * The graph is a set of (src, dst, label) triples: identical triples
//     count once, self-loops are kept, parallel edges with distinct labels
//     are distinct edges.
//   * If the empty word is in L(rho), (v, v) is a result for every start v,
//     isolated vertices included (Definition 1 ranges over V x V; the Q2
//     example of Section 1 needs c* to match the empty path).
//   * Regex syntax: '|' alternation, postfix '*', '+', '?', concatenation by
//     '.', U+00B7 or juxtaposition, parentheses.  Without a label-name table a
//     label is one lowercase letter ('a' = 0, 'b' = 1, ...); with a table a
//     label is a maximal identifier [A-Za-z0-9_]+ looked up in it.
//
// Parity status: every function here is pinned by tests in
// tests/test_oracle_pins.py (the paper's worked example of Figure 1 /
// Table 1, a second algorithm in oracle/algebra.py, closed forms and
// invariants).

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// --------------------------------------------------------------------------
// Error reporting
// --------------------------------------------------------------------------
thread_local char g_err[512];

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = -1,
  ORC_ERR_PARSE = -2,
  ORC_ERR_LABEL = -3,
  ORC_ERR_TOO_BIG = -4,
};

int fail(int code, const std::string &msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg.c_str());
  return code;
}

// --------------------------------------------------------------------------
// Regex syntax tree
// --------------------------------------------------------------------------
enum Kind { K_LABEL, K_CAT, K_ALT, K_STAR, K_PLUS, K_OPT };

struct Node {
  Kind kind;
  int label;  // K_LABEL only
  int left;   // child index
  int right;  // second child for K_CAT / K_ALT
};

struct Regex {
  std::vector<Node> nodes;
  int root = -1;
};

struct Parser {
  const std::string &s;
  size_t pos = 0;
  const std::vector<std::string> *names;  // nullptr: single letters
  Regex *re;
  int err = 0;
  std::string msg;

  Parser(const std::string &text, const std::vector<std::string> *nm, Regex *r)
      : s(text), names(nm), re(r) {}

  int add(Kind k, int label, int l, int r) {
    re->nodes.push_back(Node{k, label, l, r});
    return (int)re->nodes.size() - 1;
  }

  void skip_space() {
    while (pos < s.size() && (s[pos] == ' ' || s[pos] == '\t')) pos++;
  }

  // '.' or the two UTF-8 bytes of U+00B7 (middle dot) are explicit
  // concatenation marks.
  bool at_concat_mark() {
    if (pos < s.size() && s[pos] == '.') return true;
    if (pos + 1 < s.size() && (unsigned char)s[pos] == 0xC2 &&
        (unsigned char)s[pos + 1] == 0xB7)
      return true;
    return false;
  }
  void eat_concat_mark() { pos += (s[pos] == '.') ? 1 : 2; }

  bool at_atom_start() {
    if (pos >= s.size()) return false;
    char c = s[pos];
    if (c == '(') return true;
    if (names == nullptr) return c >= 'a' && c <= 'z';
    return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') ||
           (c >= '0' && c <= '9') || c == '_';
  }

  int set_error(int code, const std::string &m) {
    if (err == 0) {
      err = code;
      msg = m + " at position " + std::to_string(pos);
    }
    return -1;
  }

  int parse_alt() {
    int left = parse_cat();
    if (err) return -1;
    for (;;) {
      skip_space();
      if (pos < s.size() && s[pos] == '|') {
        pos++;
        int right = parse_cat();
        if (err) return -1;
        left = add(K_ALT, -1, left, right);
      } else {
        return left;
      }
    }
  }

  int parse_cat() {
    skip_space();
    int left = parse_postfix();
    if (err) return -1;
    for (;;) {
      skip_space();
      if (at_concat_mark()) {
        eat_concat_mark();
        skip_space();
        int right = parse_postfix();
        if (err) return -1;
        left = add(K_CAT, -1, left, right);
      } else if (at_atom_start()) {
        int right = parse_postfix();
        if (err) return -1;
        left = add(K_CAT, -1, left, right);
      } else {
        return left;
      }
    }
  }

  int parse_postfix() {
    int a = parse_atom();
    if (err) return -1;
    for (;;) {
      skip_space();
      if (pos >= s.size()) return a;
      char c = s[pos];
      if (c == '*') {
        pos++;
        a = add(K_STAR, -1, a, -1);
      } else if (c == '+') {
        pos++;
        a = add(K_PLUS, -1, a, -1);
      } else if (c == '?') {
        pos++;
        a = add(K_OPT, -1, a, -1);
      } else {
        return a;
      }
    }
  }

  int parse_atom() {
    skip_space();
    if (pos >= s.size()) return set_error(ORC_ERR_PARSE, "unexpected end of expression");
    char c = s[pos];
    if (c == '(') {
      pos++;
      int inner = parse_alt();
      if (err) return -1;
      skip_space();
      if (pos >= s.size() || s[pos] != ')') return set_error(ORC_ERR_PARSE, "expected ')'");
      pos++;
      return inner;
    }
    if (!at_atom_start()) return set_error(ORC_ERR_PARSE, std::string("unexpected character '") + c + "'");
    if (names == nullptr) {
      pos++;
      return add(K_LABEL, c - 'a', -1, -1);
    }
    size_t start = pos;
    while (pos < s.size() && s[pos] != '(' && at_atom_start()) pos++;
    std::string ident = s.substr(start, pos - start);
    for (size_t i = 0; i < names->size(); i++)
      if ((*names)[i] == ident) return add(K_LABEL, (int)i, -1, -1);
    pos = start;
    return set_error(ORC_ERR_LABEL, "unknown label '" + ident + "'");
  }
};

int parse_regex(const char *text, const std::vector<std::string> *names, Regex *out, std::string *msg) {
  std::string s(text ? text : "");
  Parser p(s, names, out);
  int root = p.parse_alt();
  if (!p.err) {
    p.skip_space();
    if (p.pos != s.size()) p.set_error(ORC_ERR_PARSE, "trailing characters");
  }
  if (p.err) {
    *msg = p.msg;
    return p.err;
  }
  out->root = root;
  return ORC_OK;
}

// --------------------------------------------------------------------------
// Thompson epsilon-NFA
// --------------------------------------------------------------------------
struct NFA {
  std::vector<std::vector<int>> eps;                    // epsilon moves
  std::vector<std::vector<std::pair<int, int>>> moves;  // (label, target)
  int start = -1;
  int accept = -1;

  int new_state() {
    eps.emplace_back();
    moves.emplace_back();
    return (int)eps.size() - 1;
  }
};

struct Frag {
  int in, out;
};

Frag thompson(const Regex &re, int idx, NFA &nfa) {
  const Node &n = re.nodes[idx];
  switch (n.kind) {
    case K_LABEL: {
      int a = nfa.new_state(), b = nfa.new_state();
      nfa.moves[a].push_back({n.label, b});
      return {a, b};
    }
    case K_CAT: {
      Frag x = thompson(re, n.left, nfa);
      Frag y = thompson(re, n.right, nfa);
      nfa.eps[x.out].push_back(y.in);
      return {x.in, y.out};
    }
    case K_ALT: {
      Frag x = thompson(re, n.left, nfa);
      Frag y = thompson(re, n.right, nfa);
      int a = nfa.new_state(), b = nfa.new_state();
      nfa.eps[a].push_back(x.in);
      nfa.eps[a].push_back(y.in);
      nfa.eps[x.out].push_back(b);
      nfa.eps[y.out].push_back(b);
      return {a, b};
    }
    case K_STAR: {
      Frag x = thompson(re, n.left, nfa);
      int a = nfa.new_state(), b = nfa.new_state();
      nfa.eps[a].push_back(x.in);
      nfa.eps[a].push_back(b);
      nfa.eps[x.out].push_back(x.in);
      nfa.eps[x.out].push_back(b);
      return {a, b};
    }
    case K_PLUS: {
      Frag x = thompson(re, n.left, nfa);
      int a = nfa.new_state(), b = nfa.new_state();
      nfa.eps[a].push_back(x.in);
      nfa.eps[x.out].push_back(x.in);
      nfa.eps[x.out].push_back(b);
      return {a, b};
    }
    case K_OPT: {
      Frag x = thompson(re, n.left, nfa);
      int a = nfa.new_state(), b = nfa.new_state();
      nfa.eps[a].push_back(x.in);
      nfa.eps[a].push_back(b);
      nfa.eps[x.out].push_back(b);
      return {a, b};
    }
  }
  return {-1, -1};
}

std::vector<int> closure_of(const NFA &nfa, const std::vector<int> &seed) {
  std::set<int> seen(seed.begin(), seed.end());
  std::vector<int> stack(seed.begin(), seed.end());
  while (!stack.empty()) {
    int q = stack.back();
    stack.pop_back();
    for (int r : nfa.eps[q])
      if (seen.insert(r).second) stack.push_back(r);
  }
  return std::vector<int>(seen.begin(), seen.end());
}

struct Automaton {
  NFA nfa;
  std::vector<std::vector<int>> closure;  // closure[q] = eps-closure({q})
  // Minimal partial DFA: next[d][l] = target or -1.
  int dfa_states = 0;
  int dfa_start = 0;
  std::vector<std::vector<int>> dfa_next;
  std::vector<char> dfa_final;
};

// Subset construction over the Thompson NFA, then trimming and Moore
// partition refinement.  Labels range over [0, n_labels).
int build_min_dfa(Automaton &A, int n_labels, std::string *msg) {
  const NFA &nfa = A.nfa;
  std::map<std::vector<int>, int> id;
  std::vector<std::vector<int>> sets;
  std::vector<std::vector<int>> next;
  sets.push_back(A.closure[nfa.start]);
  id[sets[0]] = 0;
  for (size_t i = 0; i < sets.size(); i++) {
    next.emplace_back(n_labels, -1);
    for (int l = 0; l < n_labels; l++) {
      std::vector<int> moved;
      for (int q : sets[i])
        for (auto &m : nfa.moves[q])
          if (m.first == l) moved.push_back(m.second);
      if (moved.empty()) continue;
      std::vector<int> T = closure_of(nfa, moved);
      auto it = id.find(T);
      int t;
      if (it == id.end()) {
        t = (int)sets.size();
        id[T] = t;
        sets.push_back(T);
        if (sets.size() > 4096) {
          *msg = "subset construction exceeded 4096 states";
          return ORC_ERR_TOO_BIG;
        }
      } else {
        t = it->second;
      }
      next[i][l] = t;
    }
  }
  int n = (int)sets.size();
  std::vector<char> fin(n, 0);
  for (int i = 0; i < n; i++)
    for (int q : sets[i])
      if (q == nfa.accept) fin[i] = 1;

  // Trim states from which no accepting state can be reached.
  std::vector<char> live(fin.begin(), fin.end());
  for (bool changed = true; changed;) {
    changed = false;
    for (int i = 0; i < n; i++) {
      if (live[i]) continue;
      for (int l = 0; l < n_labels; l++)
        if (next[i][l] >= 0 && live[next[i][l]]) {
          live[i] = 1;
          changed = true;
          break;
        }
    }
  }
  for (int i = 0; i < n; i++)
    for (int l = 0; l < n_labels; l++)
      if (next[i][l] >= 0 && !live[next[i][l]]) next[i][l] = -1;

  // Moore refinement.  Block -1 stands for the implicit dead state.
  std::vector<int> block(n);
  for (int i = 0; i < n; i++) block[i] = live[i] ? (fin[i] ? 1 : 0) : -1;
  int n_blocks = 0;
  for (;;) {
    std::map<std::vector<int>, int> sig_id;
    std::vector<int> nb(n, -1);
    for (int i = 0; i < n; i++) {
      if (block[i] < 0) continue;
      std::vector<int> sig;
      sig.push_back(block[i]);
      for (int l = 0; l < n_labels; l++) sig.push_back(next[i][l] >= 0 ? block[next[i][l]] : -1);
      auto it = sig_id.find(sig);
      if (it == sig_id.end()) {
        int b = (int)sig_id.size();
        sig_id[sig] = b;
        nb[i] = b;
      } else {
        nb[i] = it->second;
      }
    }
    int cnt = (int)sig_id.size();
    block = nb;
    if (cnt == n_blocks) break;
    n_blocks = cnt;
  }

  A.dfa_states = 0;
  A.dfa_next.clear();
  A.dfa_final.clear();
  if (block[0] < 0) {  // empty language: no live start state
    A.dfa_states = 0;
    return ORC_OK;
  }
  // Renumber blocks in breadth-first order from the start block so the
  // numbering is canonical.
  std::vector<int> order(n_blocks, -1);
  std::vector<int> rep(n_blocks, -1);
  for (int i = 0; i < n; i++)
    if (block[i] >= 0 && rep[block[i]] < 0) rep[block[i]] = i;
  std::deque<int> bq;
  int k = 0;
  order[block[0]] = k++;
  bq.push_back(block[0]);
  while (!bq.empty()) {
    int b = bq.front();
    bq.pop_front();
    int r = rep[b];
    for (int l = 0; l < n_labels; l++) {
      int t = next[r][l];
      if (t < 0) continue;
      int tb = block[t];
      if (order[tb] < 0) {
        order[tb] = k++;
        bq.push_back(tb);
      }
    }
  }
  A.dfa_states = k;
  A.dfa_start = 0;
  A.dfa_next.assign(k, std::vector<int>(n_labels, -1));
  A.dfa_final.assign(k, 0);
  for (int b = 0; b < n_blocks; b++) {
    if (order[b] < 0) continue;
    int r = rep[b];
    A.dfa_final[order[b]] = fin[r];
    for (int l = 0; l < n_labels; l++)
      if (next[r][l] >= 0) A.dfa_next[order[b]][l] = order[block[next[r][l]]];
  }
  return ORC_OK;
}

int build_automaton(const char *regex, const std::vector<std::string> *names, int n_labels, Automaton *A,
                    std::string *msg) {
  Regex re;
  int rc = parse_regex(regex, names, &re, msg);
  if (rc) return rc;
  for (auto &nd : re.nodes)
    if (nd.kind == K_LABEL && nd.label >= n_labels) n_labels = nd.label + 1;
  Frag f = thompson(re, re.root, A->nfa);
  A->nfa.start = f.in;
  A->nfa.accept = f.out;
  A->closure.resize(A->nfa.eps.size());
  for (size_t q = 0; q < A->nfa.eps.size(); q++) A->closure[q] = closure_of(A->nfa, {(int)q});
  return build_min_dfa(*A, n_labels, msg);
}

// --------------------------------------------------------------------------
// Data graph
// --------------------------------------------------------------------------
struct Graph {
  uint32_t n = 0;
  uint32_t n_labels = 0;
  uint64_t n_edges = 0;  // after removing identical triples
  // adj[v] holds (label, dst) sorted ascending.
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> adj;
  std::vector<uint8_t> vlabel;  // empty when the graph has no vertex labels
};

// Range of adj[v] entries with the given label.
inline std::pair<const std::pair<uint32_t, uint32_t> *, const std::pair<uint32_t, uint32_t> *> out_edges(
    const Graph &g, uint32_t v, uint32_t l) {
  const auto &a = g.adj[v];
  auto lo = std::lower_bound(a.begin(), a.end(), std::make_pair(l, 0u));
  auto hi = std::lower_bound(a.begin(), a.end(), std::make_pair(l + 1, 0u));
  return {a.data() + (lo - a.begin()), a.data() + (hi - a.begin())};
}

// --------------------------------------------------------------------------
// Single-source evaluation
// --------------------------------------------------------------------------

// Definition 1 for one start vertex, by BFS over (vertex, NFA state).  The
// visited set is a flag per product vertex (v, q), index v * |NFA| + q; the
// result set is a flag per vertex, read out in vertex order.
void rpq_from_nfa(const Graph &g, const Automaton &A, uint32_t s, std::vector<uint32_t> *out) {
  const size_t S = A.nfa.eps.size();
  std::vector<uint8_t> visited((size_t)g.n * S, 0);
  std::vector<uint8_t> result(g.n, 0);
  std::deque<std::pair<uint32_t, int>> queue;
  for (int q : A.closure[A.nfa.start]) {
    visited[(size_t)s * S + q] = 1;
    queue.push_back({s, q});
  }
  while (!queue.empty()) {
    auto [v, q] = queue.front();
    queue.pop_front();
    if (q == A.nfa.accept) result[v] = 1;
    for (auto &m : A.nfa.moves[q]) {
      uint32_t l = (uint32_t)m.first;
      if (l >= g.n_labels) continue;
      auto [lo, hi] = out_edges(g, v, l);
      for (auto e = lo; e != hi; ++e)
        for (int q3 : A.closure[m.second]) {
          uint8_t &seen = visited[(size_t)e->second * S + q3];
          if (!seen) {
            seen = 1;
            queue.push_back({e->second, q3});
          }
        }
    }
  }
  out->clear();
  for (uint32_t v = 0; v < g.n; v++)
    if (result[v]) out->push_back(v);
}

// Same start vertex over the minimal DFA: counts the product vertices N and
// product-edge relaxations W, and also returns the result set so the two
// automata can be checked against each other.
void rpq_from_dfa(const Graph &g, const Automaton &A, uint32_t s, std::vector<uint32_t> *out, uint64_t *W,
                  uint64_t *N) {
  *W = 0;
  *N = 0;
  out->clear();
  if (A.dfa_states == 0) return;
  const size_t S = (size_t)A.dfa_states;
  std::vector<uint8_t> visited((size_t)g.n * S, 0);
  std::vector<uint8_t> result(g.n, 0);
  std::deque<std::pair<uint32_t, int>> queue;
  visited[(size_t)s * S + A.dfa_start] = 1;
  queue.push_back({s, A.dfa_start});
  int nl = (int)A.dfa_next[0].size();
  while (!queue.empty()) {
    auto [v, q] = queue.front();
    queue.pop_front();
    *N += 1;
    if (A.dfa_final[q]) result[v] = 1;
    for (int l = 0; l < nl; l++) {
      int t = A.dfa_next[q][l];
      if (t < 0 || (uint32_t)l >= g.n_labels) continue;
      auto [lo, hi] = out_edges(g, v, (uint32_t)l);
      *W += (uint64_t)(hi - lo);
      for (auto e = lo; e != hi; ++e) {
        uint8_t &seen = visited[(size_t)e->second * S + t];
        if (!seen) {
          seen = 1;
          queue.push_back({e->second, t});
        }
      }
    }
  }
  for (uint32_t v = 0; v < g.n; v++)
    if (result[v]) out->push_back(v);
}

// --------------------------------------------------------------------------
// Result handle
// --------------------------------------------------------------------------
struct Result {
  uint32_t arity = 2;
  std::vector<uint32_t> rows;  // arity values per row
  uint64_t W = 0, N = 0;
  uint64_t automaton_mismatch = 0;  // sources where NFA and DFA sets differ
  int threads_used = 1;
};

std::vector<std::string> to_names(const char *const *names, uint32_t n) {
  std::vector<std::string> v;
  for (uint32_t i = 0; i < n; i++) v.emplace_back(names[i]);
  return v;
}

}  // namespace

// ==========================================================================
// C interface (loaded by oracle/__init__.py through ctypes)
// ==========================================================================
extern "C" {

const char *orc_last_error() { return g_err; }

int orc_graph_new(uint32_t n_vertices, uint32_t n_labels, uint64_t n_edges, const uint32_t *src,
                  const uint32_t *dst, const uint16_t *label, const uint8_t *vertex_label, void **out) {
  if (!out || (n_edges && (!src || !dst || !label))) return fail(ORC_ERR_ARG, "null argument");
  std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> t;  // (src, label, dst)
  t.reserve(n_edges);
  for (uint64_t i = 0; i < n_edges; i++) {
    if (src[i] >= n_vertices || dst[i] >= n_vertices) return fail(ORC_ERR_ARG, "vertex id out of range");
    if (label[i] >= n_labels) return fail(ORC_ERR_ARG, "edge label out of range");
    t.emplace_back(src[i], label[i], dst[i]);
  }
  std::sort(t.begin(), t.end());
  t.erase(std::unique(t.begin(), t.end()), t.end());
  Graph *g = new Graph;
  g->n = n_vertices;
  g->n_labels = n_labels;
  g->n_edges = t.size();
  g->adj.resize(n_vertices);
  for (auto &[s, l, d] : t) g->adj[s].push_back({l, d});
  if (vertex_label) g->vlabel.assign(vertex_label, vertex_label + n_vertices);
  *out = g;
  return ORC_OK;
}

void orc_graph_free(void *g) { delete (Graph *)g; }

uint64_t orc_graph_edges(void *g) { return ((Graph *)g)->n_edges; }

// Exports the minimal DFA this oracle builds: n_states, start (always 0),
// final flags and next[q * n_labels + l] (-1 for no transition).  Arrays must
// hold max_states and max_states * n_labels entries.
int orc_dfa(const char *regex, const char *const *names, uint32_t n_names, uint32_t n_labels, int max_states,
            int *n_states, uint8_t *final_flags, int32_t *next) {
  Automaton A;
  std::string msg;
  std::vector<std::string> nm = to_names(names, n_names);
  int rc = build_automaton(regex, names ? &nm : nullptr, (int)n_labels, &A, &msg);
  if (rc) return fail(rc, msg);
  *n_states = A.dfa_states;
  if (A.dfa_states > max_states) return fail(ORC_ERR_TOO_BIG, "more DFA states than the buffer holds");
  int nl = A.dfa_states ? (int)A.dfa_next[0].size() : (int)n_labels;
  for (int q = 0; q < A.dfa_states; q++) {
    final_flags[q] = (uint8_t)A.dfa_final[q];
    for (uint32_t l = 0; l < n_labels; l++) next[q * n_labels + l] = ((int)l < nl) ? A.dfa_next[q][l] : -1;
  }
  return ORC_OK;
}

// Evaluates rho from each listed start vertex (all vertices when sources is
// NULL).  Rows are the distinct (src, dst) pairs in ascending order.
int orc_rpq(void *graph, const char *regex, const char *const *names, uint32_t n_names, const uint32_t *sources,
            uint64_t n_sources, int threads, void **out) {
  Graph *g = (Graph *)graph;
  if (!g || !out) return fail(ORC_ERR_ARG, "null argument");
  Automaton A;
  std::string msg;
  std::vector<std::string> nm = to_names(names, n_names);
  int rc = build_automaton(regex, names ? &nm : nullptr, (int)g->n_labels, &A, &msg);
  if (rc) return fail(rc, msg);

  std::vector<uint32_t> srcs;
  if (sources) {
    for (uint64_t i = 0; i < n_sources; i++) {
      if (sources[i] >= g->n) return fail(ORC_ERR_ARG, "source id out of range");
      srcs.push_back(sources[i]);
    }
    std::sort(srcs.begin(), srcs.end());
    srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
  } else {
    for (uint32_t v = 0; v < g->n; v++) srcs.push_back(v);
  }

  int64_t ns = (int64_t)srcs.size();
  std::vector<std::vector<uint32_t>> per(ns);
  std::vector<uint64_t> Ws(ns, 0), Ns(ns, 0), bad(ns, 0);
  int used = 1;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
  used = threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (int64_t i = 0; i < ns; i++) {
    std::vector<uint32_t> via_dfa;
    rpq_from_nfa(*g, A, srcs[i], &per[i]);
    rpq_from_dfa(*g, A, srcs[i], &via_dfa, &Ws[i], &Ns[i]);
    bad[i] = (via_dfa != per[i]) ? 1 : 0;
  }

  Result *r = new Result;
  r->arity = 2;
  r->threads_used = used;
  size_t total = 0;
  for (auto &p : per) total += p.size();
  r->rows.reserve(2 * total);
  for (int64_t i = 0; i < ns; i++) {
    for (uint32_t d : per[i]) {
      r->rows.push_back(srcs[i]);
      r->rows.push_back(d);
    }
    r->W += Ws[i];
    r->N += Ns[i];
    r->automaton_mismatch += bad[i];
  }
  *out = r;
  return ORC_OK;
}

// Definition 2.  Atom k is atom_x[k] -regex[k]-> atom_y[k].  var_label[i] < 0
// means variable i has no label constraint.  When restrict0 is not NULL,
// variable 0 ranges only over the listed vertices (a sample).  Every variable
// must appear in at least one atom.
int orc_crpq(void *graph, uint32_t n_vars, const int32_t *var_label, uint32_t n_atoms, const uint32_t *atom_x,
             const uint32_t *atom_y, const char *const *regexes, const char *const *names, uint32_t n_names,
             const uint32_t *restrict0, uint64_t n_restrict0, int threads, void **out) {
  Graph *g = (Graph *)graph;
  if (!g || !out || n_vars == 0 || n_vars > 16) return fail(ORC_ERR_ARG, "bad argument");
  std::vector<std::string> nm = to_names(names, n_names);
  std::vector<Automaton> autos(n_atoms);
  std::vector<char> used_var(n_vars, 0);
  for (uint32_t k = 0; k < n_atoms; k++) {
    if (atom_x[k] >= n_vars || atom_y[k] >= n_vars) return fail(ORC_ERR_ARG, "atom variable out of range");
    used_var[atom_x[k]] = used_var[atom_y[k]] = 1;
    std::string msg;
    int rc = build_automaton(regexes[k], names ? &nm : nullptr, (int)g->n_labels, &autos[k], &msg);
    if (rc) return fail(rc, msg);
  }
  for (uint32_t i = 0; i < n_vars; i++)
    if (!used_var[i]) return fail(ORC_ERR_ARG, "variable appears in no atom");
  if (!g->vlabel.size())
    for (uint32_t i = 0; i < n_vars; i++)
      if (var_label && var_label[i] >= 0) return fail(ORC_ERR_ARG, "graph has no vertex labels");

  auto label_ok = [&](uint32_t var, uint32_t v) {
    return !var_label || var_label[var] < 0 || g->vlabel[v] == (uint8_t)var_label[var];
  };

  std::vector<uint32_t> first;
  if (restrict0) {
    first.assign(restrict0, restrict0 + n_restrict0);
    for (uint32_t v : first)
      if (v >= g->n) return fail(ORC_ERR_ARG, "restricted vertex out of range");
    std::sort(first.begin(), first.end());
    first.erase(std::unique(first.begin(), first.end()), first.end());
  } else {
    for (uint32_t v = 0; v < g->n; v++) first.push_back(v);
  }

  int used = 1;
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_max_threads();
  used = threads;
#endif
  std::vector<std::set<std::vector<uint32_t>>> per(first.size());

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
#endif
  for (int64_t fi = 0; fi < (int64_t)first.size(); fi++) {
    // Per-thread memo of single-source results: (atom, source) -> set.
    std::map<std::pair<uint32_t, uint32_t>, std::set<uint32_t>> memo;
    auto reach = [&](uint32_t k, uint32_t s) -> const std::set<uint32_t> & {
      auto key = std::make_pair(k, s);
      auto it = memo.find(key);
      if (it != memo.end()) return it->second;
      std::vector<uint32_t> v;
      rpq_from_nfa(*g, autos[k], s, &v);
      return memo.emplace(key, std::set<uint32_t>(v.begin(), v.end())).first->second;
    };
    std::vector<uint32_t> f(n_vars);
    // Depth-first assignment of variables 0, 1, ..., n_vars-1.
    std::vector<std::vector<uint32_t>> cand(n_vars);
    std::vector<size_t> at(n_vars, 0);
    auto candidates = [&](uint32_t i) {
      std::vector<uint32_t> c;
      if (i == 0) {
        c.push_back(first[fi]);
        return c;
      }
      for (uint32_t k = 0; k < n_atoms; k++)
        if (atom_y[k] == i && atom_x[k] < i) {
          const auto &r = reach(k, f[atom_x[k]]);
          c.assign(r.begin(), r.end());
          return c;
        }
      for (uint32_t v = 0; v < g->n; v++) c.push_back(v);
      return c;
    };
    auto consistent = [&](uint32_t i) {
      if (!label_ok(i, f[i])) return false;
      for (uint32_t k = 0; k < n_atoms; k++) {
        uint32_t x = atom_x[k], y = atom_y[k];
        if (x > i || y > i || (x != i && y != i)) continue;
        const auto &r = reach(k, f[x]);
        if (!r.count(f[y])) return false;
      }
      return true;
    };
    int64_t i = 0;
    cand[0] = candidates(0);
    at[0] = 0;
    while (i >= 0) {
      if (at[i] >= cand[i].size()) {
        i--;
        if (i >= 0) at[i]++;
        continue;
      }
      f[i] = cand[i][at[i]];
      if (!consistent((uint32_t)i)) {
        at[i]++;
        continue;
      }
      if (i == (int64_t)n_vars - 1) {
        per[fi].insert(f);
        at[i]++;
        continue;
      }
      i++;
      cand[i] = candidates((uint32_t)i);
      at[i] = 0;
    }
  }

  Result *r = new Result;
  r->arity = n_vars;
  r->threads_used = used;
  for (auto &s : per)
    for (auto &t : s)
      for (uint32_t x : t) r->rows.push_back(x);
  *out = r;
  return ORC_OK;
}

uint64_t orc_result_rows(void *r) {
  Result *x = (Result *)r;
  return x->rows.size() / x->arity;
}
uint32_t orc_result_arity(void *r) { return ((Result *)r)->arity; }
void orc_result_copy(void *r, uint32_t *out) {
  Result *x = (Result *)r;
  if (!x->rows.empty()) std::memcpy(out, x->rows.data(), x->rows.size() * sizeof(uint32_t));
}
void orc_result_work(void *r, uint64_t *W, uint64_t *N, uint64_t *mismatch, int *threads) {
  Result *x = (Result *)r;
  *W = x->W;
  *N = x->N;
  *mismatch = x->automaton_mismatch;
  *threads = x->threads_used;
}
void orc_result_free(void *r) { delete (Result *)r; }

}  // extern "C"
