// Regex -> minimal DFA, on the host (the query-interpretation step of the
// paper's architecture, Section 7, which builds the automata-based plan of
// Section 2.2; the plans of Section 4.1 use the minimal DFA, e.g. abc* as
// q0 -a-> q1 -b-> q2 with a c self-loop on the accepting q2).
//
// Pipeline: tokenizer -> precedence-climbing parser -> Glushkov (position)
// automaton -> subset construction -> Hopcroft minimization of the completed
// DFA -> removal of the dead class -> breadth-first canonical numbering.
// The result is the unique minimal partial DFA of L(rho), so its states and
// transition table do not depend on how the expression was written.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "rpq_internal.h"

namespace rpq {
namespace {

enum TokKind { T_LABEL, T_BAR, T_STAR, T_PLUS, T_QMARK, T_LPAR, T_RPAR, T_DOT, T_END };

struct Token {
  TokKind kind;
  int label;
  size_t pos;
};

bool ident_char(char c) {
  return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_';
}

int tokenize(const std::string &s, const char *const *names, uint32_t n_names, std::vector<Token> *out,
             std::string *msg) {
  size_t i = 0;
  while (i < s.size()) {
    char c = s[i];
    if (c == ' ' || c == '\t') {
      i++;
      continue;
    }
    Token t{T_END, -1, i};
    if (c == '|') {
      t.kind = T_BAR;
      i++;
    } else if (c == '*') {
      t.kind = T_STAR;
      i++;
    } else if (c == '+') {
      t.kind = T_PLUS;
      i++;
    } else if (c == '?') {
      t.kind = T_QMARK;
      i++;
    } else if (c == '(') {
      t.kind = T_LPAR;
      i++;
    } else if (c == ')') {
      t.kind = T_RPAR;
      i++;
    } else if (c == '.') {
      t.kind = T_DOT;
      i++;
    } else if ((unsigned char)c == 0xC2 && i + 1 < s.size() && (unsigned char)s[i + 1] == 0xB7) {
      t.kind = T_DOT;
      i += 2;
    } else if (names == nullptr && c >= 'a' && c <= 'z') {
      t.kind = T_LABEL;
      t.label = c - 'a';
      i++;
    } else if (names != nullptr && ident_char(c)) {
      size_t j = i;
      while (j < s.size() && ident_char(s[j])) j++;
      std::string id = s.substr(i, j - i);
      int found = -1;
      for (uint32_t k = 0; k < n_names; k++)
        if (names[k] && id == names[k]) {
          found = (int)k;
          break;
        }
      if (found < 0) {
        *msg = "unknown label '" + id + "' at position " + std::to_string(i);
        return RPQ_ERR_UNKNOWN_LABEL;
      }
      t.kind = T_LABEL;
      t.label = found;
      i = j;
    } else {
      *msg = std::string("unexpected character '") + c + "' at position " + std::to_string(i);
      return RPQ_ERR_PARSE;
    }
    out->push_back(t);
  }
  out->push_back(Token{T_END, -1, s.size()});
  return RPQ_OK;
}

// Syntax tree with Glushkov attributes computed bottom-up as nodes are built.
struct GNode {
  bool nullable;
  uint64_t first, last;  // position sets (bit p = position p, p >= 1)
};

struct Glushkov {
  std::vector<uint64_t> follow;  // follow[p]
  std::vector<int> pos_label;    // pos_label[p]
  int positions = 0;
  bool overflow = false;

  GNode leaf(int label) {
    if (positions >= RPQ_MAX_POSITIONS) {
      overflow = true;
      return GNode{false, 0, 0};
    }
    int p = ++positions;
    if ((int)follow.size() <= p) {
      follow.resize(p + 1, 0);
      pos_label.resize(p + 1, -1);
    }
    pos_label[p] = label;
    return GNode{false, 1ull << p, 1ull << p};
  }
  void link(uint64_t from, uint64_t to) {
    for (int p = 1; p <= positions; p++)
      if (from >> p & 1) follow[p] |= to;
  }
  GNode cat(const GNode &a, const GNode &b) {
    link(a.last, b.first);
    return GNode{a.nullable && b.nullable, a.first | (a.nullable ? b.first : 0), b.last | (b.nullable ? a.last : 0)};
  }
  GNode alt(const GNode &a, const GNode &b) {
    return GNode{a.nullable || b.nullable, a.first | b.first, a.last | b.last};
  }
  GNode star(const GNode &a) {
    link(a.last, a.first);
    return GNode{true, a.first, a.last};
  }
  GNode plus(const GNode &a) {
    link(a.last, a.first);
    return GNode{a.nullable, a.first, a.last};
  }
  GNode opt(const GNode &a) { return GNode{true, a.first, a.last}; }
};

struct Parser {
  const std::vector<Token> &tok;
  size_t at = 0;
  Glushkov &gl;
  int err = RPQ_OK;
  std::string msg;

  Parser(const std::vector<Token> &t, Glushkov &g) : tok(t), gl(g) {}

  const Token &peek() const { return tok[at]; }
  bool fail(const char *what) {
    if (err == RPQ_OK) {
      err = RPQ_ERR_PARSE;
      msg = std::string(what) + " at position " + std::to_string(peek().pos);
    }
    return false;
  }
  static bool starts_atom(TokKind k) { return k == T_LABEL || k == T_LPAR; }

  // expr := seq ('|' seq)*
  bool expr(GNode *out) {
    GNode acc;
    if (!seq(&acc)) return false;
    while (peek().kind == T_BAR) {
      at++;
      GNode rhs;
      if (!seq(&rhs)) return false;
      acc = gl.alt(acc, rhs);
    }
    *out = acc;
    return true;
  }
  // seq := item (('.' item) | item)*
  bool seq(GNode *out) {
    GNode acc;
    if (!item(&acc)) return false;
    for (;;) {
      TokKind k = peek().kind;
      if (k == T_DOT) {
        at++;
      } else if (!starts_atom(k)) {
        break;
      }
      GNode rhs;
      if (!item(&rhs)) return false;
      acc = gl.cat(acc, rhs);
    }
    *out = acc;
    return true;
  }
  // item := primary ('*' | '+' | '?')*
  bool item(GNode *out) {
    GNode a;
    if (!primary(&a)) return false;
    for (;;) {
      TokKind k = peek().kind;
      if (k == T_STAR)
        a = gl.star(a);
      else if (k == T_PLUS)
        a = gl.plus(a);
      else if (k == T_QMARK)
        a = gl.opt(a);
      else
        break;
      at++;
    }
    *out = a;
    return true;
  }
  bool primary(GNode *out) {
    const Token &t = peek();
    if (t.kind == T_LABEL) {
      at++;
      *out = gl.leaf(t.label);
      return true;
    }
    if (t.kind == T_LPAR) {
      at++;
      if (!expr(out)) return false;
      if (peek().kind != T_RPAR) return fail("expected ')'");
      at++;
      return true;
    }
    if (t.kind == T_END) return fail("unexpected end of expression");
    return fail("unexpected token");
  }
};

// Hopcroft's partition refinement on a complete DFA with N states over an
// alphabet of A symbols.  Returns the class of every state.
std::vector<int> hopcroft(int N, int A, const std::vector<int> &delta, const std::vector<char> &accepting) {
  // inverse transitions
  std::vector<std::vector<int>> inv((size_t)N * A);
  for (int s = 0; s < N; s++)
    for (int c = 0; c < A; c++) inv[(size_t)delta[(size_t)s * A + c] * A + c].push_back(s);

  std::vector<int> cls(N);
  std::vector<std::vector<int>> members;
  std::vector<int> acc, rej;
  for (int s = 0; s < N; s++) (accepting[s] ? acc : rej).push_back(s);
  for (auto *grp : {&acc, &rej})
    if (!grp->empty()) {
      for (int s : *grp) cls[s] = (int)members.size();
      members.push_back(*grp);
    }
  std::vector<std::vector<char>> waiting(members.size(), std::vector<char>(A, 0));
  std::deque<std::pair<int, int>> work;
  if (members.size() == 2) {
    int small = members[0].size() <= members[1].size() ? 0 : 1;
    for (int c = 0; c < A; c++) {
      work.push_back({small, c});
      waiting[small][c] = 1;
    }
  }
  std::vector<char> mark(N, 0);
  std::vector<int> touched_count;
  while (!work.empty()) {
    auto [b, c] = work.front();
    work.pop_front();
    waiting[b][c] = 0;
    // X = predecessors of class b on symbol c
    std::vector<int> X;
    for (int t : members[b])
      for (int s : inv[(size_t)t * A + c]) X.push_back(s);
    if (X.empty()) continue;
    for (int s : X) mark[s] = 1;
    std::vector<int> classes;
    for (int s : X) classes.push_back(cls[s]);
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int y : classes) {
      std::vector<int> in, out;
      for (int s : members[y]) (mark[s] ? in : out).push_back(s);
      if (in.empty() || out.empty()) continue;
      int z = (int)members.size();
      members[y] = in;
      members.push_back(out);
      for (int s : out) cls[s] = z;
      waiting.push_back(std::vector<char>(A, 0));
      for (int cc = 0; cc < A; cc++) {
        if (waiting[y][cc]) {
          waiting[z][cc] = 1;
          work.push_back({z, cc});
        } else {
          int pick = members[y].size() <= members[z].size() ? y : z;
          waiting[pick][cc] = 1;
          work.push_back({pick, cc});
        }
      }
    }
    for (int s : X) mark[s] = 0;
  }
  return cls;
}

// Completes a partial DFA (n states, A symbols, raw[s * A + c] = target or -1,
// state 0 the start) with a dead state, minimizes it, drops the dead class
// and numbers the classes breadth-first from the start (symbols ascending),
// which makes the table canonical.  Fills the kernel descriptor.
int finish_dfa(int n, int A, const std::vector<int> &raw, const std::vector<char> &acc_raw, QueryDesc *out,
               std::vector<int32_t> *next_out, std::string *msg) {
  int N = n + 1, dead = n;
  std::vector<int> delta((size_t)N * A, dead);
  std::vector<char> accepting(N, 0);
  for (int s = 0; s < n; s++) {
    accepting[s] = acc_raw[s];
    for (int c = 0; c < A; c++)
      if (raw[(size_t)s * A + c] >= 0) delta[(size_t)s * A + c] = raw[(size_t)s * A + c];
  }
  std::vector<int> cls = hopcroft(N, A, delta, accepting);
  int dead_cls = cls[dead];

  std::map<int, int> num;
  std::vector<int> rep;  // representative raw state of each numbered class
  if (cls[0] != dead_cls) {
    std::deque<int> bfs;
    num[cls[0]] = 0;
    rep.push_back(0);
    bfs.push_back(0);
    while (!bfs.empty()) {
      int r = bfs.front();
      bfs.pop_front();
      for (int c = 0; c < A; c++) {
        int t = delta[(size_t)r * A + c];
        int tc = cls[t];
        if (tc == dead_cls || num.count(tc)) continue;
        num[tc] = (int)rep.size();
        rep.push_back(t);
        bfs.push_back(t);
      }
    }
  }
  int Q = (int)rep.size();
  if (Q > RPQ_MAX_STATES) {
    *msg = "minimal DFA has " + std::to_string(Q) + " states (limit " + std::to_string(RPQ_MAX_STATES) + ")";
    return RPQ_ERR_TOO_COMPLEX;
  }
  std::vector<int32_t> next((size_t)Q * A, -1);
  uint32_t fmask = 0;
  for (int q = 0; q < Q; q++) {
    if (accepting[rep[q]]) fmask |= 1u << q;
    for (int c = 0; c < A; c++) {
      int tc = cls[delta[(size_t)rep[q] * A + c]];
      if (tc != dead_cls) next[(size_t)q * A + c] = num[tc];
    }
  }
  QueryDesc d;
  std::memset(&d, 0, sizeof(d));
  d.n_states = (uint32_t)Q;
  d.final_mask = fmask;
  d.n_labels = (uint32_t)A;
  int nt = 0;
  for (int q = 0; q < Q; q++) {
    d.out_begin[q] = (uint16_t)nt;
    for (int c = 0; c < A; c++) {
      int t = next[(size_t)q * A + c];
      if (t < 0) continue;
      if (nt >= RPQ_MAX_TRANSITIONS) {
        *msg = "too many DFA transitions";
        return RPQ_ERR_TOO_COMPLEX;
      }
      d.out_label[nt] = (uint8_t)c;
      d.out_to[nt] = (uint8_t)t;
      nt++;
    }
  }
  for (int q = Q; q <= RPQ_MAX_STATES; q++) d.out_begin[q] = (uint16_t)nt;
  d.n_trans = (uint32_t)nt;
  int ng = 0;
  for (int q2 = 0; q2 < Q; q2++) {
    d.in_begin[q2] = (uint16_t)ng;
    for (int c = 0; c < A; c++) {
      uint32_t from = 0;
      for (int q = 0; q < Q; q++)
        if (next[(size_t)q * A + c] == q2) from |= 1u << q;
      if (!from) continue;
      d.in_label[ng] = (uint8_t)c;
      d.in_from[ng] = from;
      ng++;
    }
  }
  for (int q = Q; q <= RPQ_MAX_STATES; q++) d.in_begin[q] = (uint16_t)ng;
  *out = d;
  *next_out = next;
  return RPQ_OK;
}

}  // namespace

int compile_regex(const char *regex, const char *const *names, uint32_t n_names, HostQuery *out, std::string *msg) {
  if (!regex || !out) {
    *msg = "null argument";
    return RPQ_ERR_INVALID_ARG;
  }
  std::vector<Token> toks;
  int rc = tokenize(regex, names, n_names, &toks, msg);
  if (rc) return rc;
  Glushkov gl;
  Parser ps(toks, gl);
  GNode root;
  bool ok = ps.expr(&root);
  if (ok && ps.peek().kind != T_END) ok = ps.fail("trailing input");
  if (!ok) {
    *msg = ps.msg;
    return ps.err;
  }
  if (gl.overflow) {
    *msg = "more than " + std::to_string(RPQ_MAX_POSITIONS) + " label occurrences";
    return RPQ_ERR_TOO_COMPLEX;
  }
  int A = 0;
  for (int p = 1; p <= gl.positions; p++) A = std::max(A, gl.pos_label[p] + 1);
  if (A > RPQ_MAX_LABELS) {
    *msg = "label id beyond RPQ_MAX_LABELS";
    return RPQ_ERR_TOO_COMPLEX;
  }
  if (A == 0) A = 1;

  // Subset construction over Glushkov states {0 (initial)} U positions.
  auto step = [&](uint64_t S, int c) {
    uint64_t T = 0;
    for (int p = 0; p <= gl.positions; p++) {
      if (!(S >> p & 1)) continue;
      uint64_t succ = (p == 0) ? root.first : gl.follow[p];
      for (int r = 1; r <= gl.positions; r++)
        if ((succ >> r & 1) && gl.pos_label[r] == c) T |= 1ull << r;
    }
    return T;
  };
  const uint64_t accept_set = root.last | (root.nullable ? 1ull : 0ull);
  std::map<uint64_t, int> index;
  std::vector<uint64_t> sets{1ull};
  index[1ull] = 0;
  std::vector<int> raw;  // raw[s * A + c], -1 none
  for (size_t i = 0; i < sets.size(); i++) {
    for (int c = 0; c < A; c++) {
      uint64_t T = step(sets[i], c);
      int t = -1;
      if (T) {
        auto it = index.find(T);
        if (it == index.end()) {
          t = (int)sets.size();
          index[T] = t;
          sets.push_back(T);
          if (sets.size() > 4096) {
            *msg = "subset construction exceeded 4096 states";
            return RPQ_ERR_TOO_COMPLEX;
          }
        } else {
          t = it->second;
        }
      }
      raw.push_back(t);
    }
  }
  std::vector<char> acc_raw(sets.size(), 0);
  for (size_t k = 0; k < sets.size(); k++) acc_raw[k] = (sets[k] & accept_set) != 0;
  HostQuery hq;
  rc = finish_dfa((int)sets.size(), A, raw, acc_raw, &hq.d, &hq.next, msg);
  if (rc) return rc;

  // The reversed language (for evaluation from the target end over in-edges):
  // subset construction over the reversed minimal DFA, starting from its
  // accepting states; a set accepts when it holds the forward start state.
  hq.has_rev = false;
  std::memset(&hq.rev, 0, sizeof(hq.rev));
  const int Q = (int)hq.d.n_states;
  if (Q > 0) {
    std::map<uint32_t, int> rindex;
    std::vector<uint32_t> rsets{hq.d.final_mask};
    rindex[hq.d.final_mask] = 0;
    std::vector<int> rraw;
    bool too_big = false;
    for (size_t k = 0; k < rsets.size() && !too_big; k++) {
      for (int c = 0; c < A; c++) {
        uint32_t T = 0;
        for (int q = 0; q < Q; q++) {
          int t = hq.next[(size_t)q * A + c];
          if (t >= 0 && (rsets[k] >> t & 1u)) T |= 1u << q;
        }
        int id = -1;
        if (T) {
          auto it = rindex.find(T);
          if (it == rindex.end()) {
            id = (int)rsets.size();
            rindex[T] = id;
            rsets.push_back(T);
            if (rsets.size() > 4096) too_big = true;
          } else {
            id = it->second;
          }
        }
        rraw.push_back(id);
      }
    }
    if (!too_big) {
      std::vector<char> racc(rsets.size(), 0);
      for (size_t k = 0; k < rsets.size(); k++) racc[k] = (rsets[k] & 1u) != 0;
      std::string rmsg;
      if (finish_dfa((int)rsets.size(), A, rraw, racc, &hq.rev, &hq.rev_next, &rmsg) == RPQ_OK) hq.has_rev = true;
    }
  }
  *out = hq;
  return RPQ_OK;
}

// The minimal DFA of L(alpha) . x for a label x that alpha does not use: from
// every accepting state of alpha an x-edge leads to one new accepting state,
// and alpha's own accepting states stop accepting.
int dfa_then_label(const HostQuery &alpha, uint32_t x, HostQuery *out, std::string *msg) {
  const int Q = (int)alpha.d.n_states;
  const int A0 = (int)alpha.d.n_labels;
  if ((int)x < A0 || x >= RPQ_MAX_LABELS) {
    *msg = "the extra label must be above alpha's labels and below RPQ_MAX_LABELS";
    return RPQ_ERR_INVALID_ARG;
  }
  const int A = (int)x + 1, F = Q;
  std::vector<int> raw((size_t)(Q + 1) * A, -1);
  std::vector<char> acc(Q + 1, 0);
  for (int q = 0; q < Q; q++) {
    for (int c = 0; c < A0; c++) raw[(size_t)q * A + c] = alpha.next[(size_t)q * A0 + c];
    if ((alpha.d.final_mask >> q) & 1u) raw[(size_t)q * A + x] = F;
  }
  acc[F] = 1;
  HostQuery hq;
  hq.has_rev = false;
  const int rc = finish_dfa(Q + 1, A, raw, acc, &hq.d, &hq.next, msg);
  if (rc == RPQ_OK) *out = hq;
  return rc;
}

}  // namespace rpq
