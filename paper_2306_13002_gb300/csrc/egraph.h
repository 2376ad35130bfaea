// E-graph of the host rewriter: hash-consed e-nodes over union-find e-classes, congruence
// rebuild, the rewrite-rule families and bottom-up extraction under the paper's cost model
// (Sec. IV-V). Host-only C++ shared by the two generators of rewriter.cu (per-iteration loop
// bodies) and rewriter_march.cu (cross-iteration march kernels).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <tuple>
#include <unordered_map>
#include <utility>
#include <vector>

namespace acs {
namespace rw {

// FLUX: a neighbour's flux value read by the march kernel (payload d * 8 + (c - 1) * 2 + side,
// side 0 = +e_d, 1 = -e_d), a leaf of the cross-iteration combine body.
enum Op : int { CONST = 0, PARAM, LOAD, ADD, SUB, MUL, DIV, FMA, NEG, RCP, FLUX, NOPS };
static const char* kOpName[NOPS] = {"const", "param", "load", "add", "sub", "mul", "div", "fma", "neg", "rcp",
                                    "flux"};
inline int arity(int op) {
    switch (op) {
        case CONST: case PARAM: case LOAD: case FLUX: return 0;
        case NEG: case RCP: return 1;
        case FMA: return 3;
        default: return 2;
    }
}

// Parameters of the generated kernel (q[] array).
enum Param : int { P_GAMMA = 0, P_EPS = 1, P_HX = 2, P_HY = 3, P_HZ = 4, P_ONE = 5, P_MONE = 6, P_NZ = 7 };

struct Node {
    int op;
    int a, b, c;        // child e-classes (canonical after rebuild)
    int64_t payload;    // CONST: double bits; PARAM: index; LOAD: comp * 13 + point
};

// Counter-based random stream (SplitMix64 mixing of seed + (counter+1) * golden ratio).
struct Rng {
    uint64_t seed, ctr = 0;
    explicit Rng(uint64_t s) : seed(s) {}
    uint64_t next() {
        uint64_t z = seed + (++ctr) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    int below(int n) { return (int)(next() % (uint64_t)n); }
};

struct Key {
    int op, a, b, c;
    int64_t payload;
    bool operator==(const Key& o) const { return op == o.op && a == o.a && b == o.b && c == o.c && payload == o.payload; }
};
struct KeyHash {
    size_t operator()(const Key& k) const {
        uint64_t h = (uint64_t)k.op * 0x9E3779B97F4A7C15ULL;
        h ^= (uint64_t)(uint32_t)k.a + 0x85EBCA6B + (h << 6) + (h >> 2);
        h ^= (uint64_t)(uint32_t)k.b + 0xC2B2AE35 + (h << 6) + (h >> 2);
        h ^= (uint64_t)(uint32_t)k.c + 0x27D4EB2F + (h << 6) + (h >> 2);
        h ^= (uint64_t)k.payload + 0x165667B1 + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};

class EGraph {
   public:
    std::vector<Node> nodes;
    std::vector<int> node_class;  // class id (not necessarily canonical) of each node
    std::vector<int> parent;      // union-find over class ids
    std::unordered_map<Key, int, KeyHash> memo;
    int nclasses = 0;

    int find(int x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    }
    Key key_of(const Node& n) {
        const int ar = arity(n.op);
        return Key{n.op, ar > 0 ? find(n.a) : -1, ar > 1 ? find(n.b) : -1, ar > 2 ? find(n.c) : -1, n.payload};
    }
    int add(int op, int a = -1, int b = -1, int c = -1, int64_t payload = 0) {
        Node n{op, a, b, c, payload};
        Key k = key_of(n);
        auto it = memo.find(k);
        if (it != memo.end()) return find(node_class[it->second]);
        n.a = k.a;
        n.b = k.b;
        n.c = k.c;
        nodes.push_back(n);
        const int cls = nclasses++;
        parent.push_back(cls);
        node_class.push_back(cls);
        memo.emplace(k, (int)nodes.size() - 1);
        return cls;
    }
    int cnst(double v) {
        int64_t bits;
        std::memcpy(&bits, &v, 8);
        return add(CONST, -1, -1, -1, bits);
    }
    bool merge(int x, int y) {
        x = find(x);
        y = find(y);
        if (x == y) return false;
        if (x > y) std::swap(x, y);
        parent[y] = x;
        return true;
    }
    // Restore the congruence invariant: nodes with equal canonical keys share a class.
    void rebuild() {
        for (int pass = 0; pass < 64; ++pass) {
            std::unordered_map<Key, int, KeyHash> m;
            m.reserve(nodes.size() * 2);
            bool changed = false;
            for (size_t i = 0; i < nodes.size(); ++i) {
                Key k = key_of(nodes[i]);
                auto it = m.find(k);
                if (it == m.end())
                    m.emplace(k, (int)i);
                else if (merge(node_class[it->second], node_class[i]))
                    changed = true;
            }
            if (!changed) {
                memo.swap(m);
                for (auto& n : nodes) {
                    const int ar = arity(n.op);
                    if (ar > 0) n.a = find(n.a);
                    if (ar > 1) n.b = find(n.b);
                    if (ar > 2) n.c = find(n.c);
                }
                return;
            }
        }
    }
    // nodes of each canonical class
    std::vector<std::vector<int>> class_nodes() {
        std::vector<std::vector<int>> cn(nclasses);
        for (size_t i = 0; i < nodes.size(); ++i) cn[find(node_class[i])].push_back((int)i);
        return cn;
    }
    bool const_value(const std::vector<std::vector<int>>& cn, int cls, double* v) {
        for (int ni : cn[find(cls)])
            if (nodes[ni].op == CONST) {
                std::memcpy(v, &nodes[ni].payload, 8);
                return true;
            }
        return false;
    }
};

// ------------------------------------------------------------------ rules

// The first seven families are the paper's (Table I, constant folding, and the division,
// distributivity and subtraction/negation families it can express but disables, Sec. V-A).
// F_COLLECT is this library's: like-term collection of a whole sum, an identity over the reals
// that computer-algebra systems apply as a normal form; an equality-saturation schedule reaches
// it only through a combinatorial number of ASSOC/COMM steps.
// F_EXPAND (distributive expansion, the direction of distributivity the factoring rules of
// F_DISTRIB do not take) and F_NEGPUSH (negation moved into products, sums and FMAs: -(a b) =
// (-a) b, -(a b + c) = (-a) b + (-c), -(a + b) = (-a) - b, -(a - b) = b - a) are also this
// library's; both are identities over the reals and exact in IEEE arithmetic for negation.
enum Family : int { F_FMA = 0, F_COMM, F_ASSOC, F_FOLD, F_DIV, F_DISTRIB, F_SUBNEG, F_COLLECT, F_EXPAND, F_NEGPUSH,
                    NFAM };
constexpr int NFAM_PAPER = F_COLLECT;

// Exact constant folding only: the folded double must equal the exact result.
inline bool exact_add(double a, double b, double* r) {
    const double s = a + b, bb = s - a, err = (a - (s - bb)) + (b - bb);
    *r = s;
    return err == 0.0 && std::isfinite(s);
}
inline bool exact_mul(double a, double b, double* r) {
    const double p = a * b;
    *r = p;
    return std::fma(a, b, -p) == 0.0 && std::isfinite(p);
}

struct Pending {
    int cls;       // e-class the new expression joins
    int op, a, b, c;
    int64_t payload;
    int inner_op = -1, ia = -1, ib = -1;  // optional child built first, placed in slot inner_slot
    int inner_slot = -1;
    int inner2_op = -1, ja = -1, jb = -1;  // an optional second such child, in slot inner2_slot
    int inner2_slot = -1;
};

class Rewriter {
   public:
    EGraph& g;
    explicit Rewriter(EGraph& eg) : g(eg) {}

    // Collect the matches of one family over all e-nodes.
    void match(int fam, const std::vector<std::vector<int>>& cn, std::vector<Pending>& out, std::vector<int>& unions) {
        auto has = [&](int cls, int op, std::vector<const Node*>& found) {
            found.clear();
            for (int ni : cn[g.find(cls)])
                if (g.nodes[ni].op == op) found.push_back(&g.nodes[ni]);
            return !found.empty();
        };
        std::vector<const Node*> f1, f2;
        const size_t nn = g.nodes.size();
        for (size_t i = 0; i < nn; ++i) {
            const Node n = g.nodes[i];
            const int cls = g.find(g.node_class[i]);
            switch (fam) {
                case F_FMA:
                    if (n.op == ADD) {
                        for (int side = 0; side < 2; ++side) {
                            const int x = side ? n.a : n.b, other = side ? n.b : n.a;
                            if (has(x, MUL, f1))
                                for (auto* m : f1) out.push_back({cls, FMA, m->a, m->b, other, 0});
                        }
                    } else if (n.op == SUB) {
                        if (has(n.b, MUL, f1))  // A - B*C -> FMA(-B, C, A)
                            for (auto* m : f1) {
                                Pending p{cls, FMA, -2, m->b, n.a, 0};
                                p.inner_op = NEG, p.ia = m->a, p.inner_slot = 0;
                                out.push_back(p);
                            }
                        if (has(n.a, MUL, f1))  // B*C - A -> FMA(B, C, -A)
                            for (auto* m : f1) {
                                Pending p{cls, FMA, m->a, m->b, -2, 0};
                                p.inner_op = NEG, p.ia = n.b, p.inner_slot = 2;
                                out.push_back(p);
                            }
                    }
                    break;
                case F_COMM:
                    if (n.op == ADD || n.op == MUL) out.push_back({cls, n.op, n.b, n.a, -1, 0});
                    break;
                case F_ASSOC:
                    if (n.op == ADD || n.op == MUL) {
                        if (has(n.b, n.op, f1))  // A op (B op C) -> (A op B) op C
                            for (auto* m : f1) {
                                Pending p{cls, n.op, -2, m->b, -1, 0};
                                p.inner_op = n.op, p.ia = n.a, p.ib = m->a, p.inner_slot = 0;
                                out.push_back(p);
                            }
                        if (has(n.a, n.op, f1))  // (A op B) op C -> A op (B op C)
                            for (auto* m : f1) {
                                Pending p{cls, n.op, m->a, -2, -1, 0};
                                p.inner_op = n.op, p.ia = m->b, p.ib = n.b, p.inner_slot = 1;
                                out.push_back(p);
                            }
                    }
                    break;
                case F_FOLD: {
                    double x, y, r;
                    if ((n.op == ADD || n.op == SUB || n.op == MUL) && g.const_value(cn, n.a, &x) &&
                        g.const_value(cn, n.b, &y)) {
                        const bool ok = n.op == MUL ? exact_mul(x, y, &r) : exact_add(x, n.op == SUB ? -y : y, &r);
                        if (ok) {
                            int64_t bits;
                            std::memcpy(&bits, &r, 8);
                            out.push_back({cls, CONST, -1, -1, -1, bits});
                        }
                    } else if (n.op == NEG && g.const_value(cn, n.a, &x)) {
                        r = -x;
                        int64_t bits;
                        std::memcpy(&bits, &r, 8);
                        out.push_back({cls, CONST, -1, -1, -1, bits});
                    } else if (n.op == ADD) {
                        if (g.const_value(cn, n.b, &y) && y == 0.0 && !std::signbit(y)) unions.push_back(cls), unions.push_back(n.a);
                        if (g.const_value(cn, n.a, &x) && x == 0.0 && !std::signbit(x)) unions.push_back(cls), unions.push_back(n.b);
                    } else if (n.op == MUL) {
                        if (g.const_value(cn, n.b, &y) && y == 1.0) unions.push_back(cls), unions.push_back(n.a);
                        if (g.const_value(cn, n.a, &x) && x == 1.0) unions.push_back(cls), unions.push_back(n.b);
                    }
                    break;
                }
                case F_DIV:
                    if (n.op == DIV) {  // A / B -> A * rcp(B)
                        Pending p{cls, MUL, n.a, -2, -1, 0};
                        p.inner_op = RCP, p.ia = n.b, p.inner_slot = 1;
                        out.push_back(p);
                        if (has(n.a, MUL, f1))  // (A*B)/C -> A * (B/C)
                            for (auto* m : f1) {
                                Pending q{cls, MUL, m->a, -2, -1, 0};
                                q.inner_op = DIV, q.ia = m->b, q.ib = n.b, q.inner_slot = 1;
                                out.push_back(q);
                            }
                    } else if (n.op == MUL && has(n.b, DIV, f1)) {  // A * (B/C) -> (A*B)/C
                        for (auto* m : f1) {
                            Pending q{cls, DIV, -2, m->b, -1, 0};
                            q.inner_op = MUL, q.ia = n.a, q.ib = m->a, q.inner_slot = 0;
                            out.push_back(q);
                        }
                    }
                    break;
                case F_DISTRIB:
                    if ((n.op == ADD || n.op == SUB) && has(n.a, MUL, f1) && has(n.b, MUL, f2)) {
                        // A*B +- A*C -> A * (B +- C)  (common left factor, same e-class)
                        for (auto* m1 : f1)
                            for (auto* m2 : f2) {
                                if (g.find(m1->a) == g.find(m2->a)) {
                                    Pending p{cls, MUL, m1->a, -2, -1, 0};
                                    p.inner_op = n.op, p.ia = m1->b, p.ib = m2->b, p.inner_slot = 1;
                                    out.push_back(p);
                                }
                                if (g.find(m1->b) == g.find(m2->b)) {
                                    Pending p{cls, MUL, -2, m1->b, -1, 0};
                                    p.inner_op = n.op, p.ia = m1->a, p.ib = m2->a, p.inner_slot = 0;
                                    out.push_back(p);
                                }
                            }
                    }
                    break;
                case F_SUBNEG:
                    if (n.op == SUB) {  // A - B -> A + (-B)
                        Pending p{cls, ADD, n.a, -2, -1, 0};
                        p.inner_op = NEG, p.ia = n.b, p.inner_slot = 1;
                        out.push_back(p);
                    } else if (n.op == ADD && has(n.b, NEG, f1)) {  // A + (-B) -> A - B
                        for (auto* m : f1) out.push_back({cls, SUB, n.a, m->a, -1, 0});
                    } else if (n.op == NEG && has(n.a, NEG, f1)) {  // -(-A) -> A
                        for (auto* m : f1) unions.push_back(cls), unions.push_back(m->a);
                    }
                    break;
                case F_EXPAND:
                    if (n.op == MUL) {
                        for (int side = 0; side < 2; ++side) {   // A * (X1 +- X2), (X1 +- X2) * A
                            const int x = side ? n.a : n.b, A = side ? n.b : n.a;
                            for (int sop : {ADD, SUB})
                                if (has(x, sop, f1))
                                    for (auto* m : f1) {
                                        Pending p{cls, sop, -2, -2, -1, 0};
                                        p.inner_op = MUL, p.ia = A, p.ib = m->a, p.inner_slot = 0;
                                        p.inner2_op = MUL, p.ja = A, p.jb = m->b, p.inner2_slot = 1;
                                        out.push_back(p);
                                    }
                        }
                    }
                    break;
                case F_NEGPUSH:
                    if (n.op == NEG) {
                        if (has(n.a, MUL, f1))   // -(A B) -> (-A) B
                            for (auto* m : f1) {
                                Pending p{cls, MUL, -2, m->b, -1, 0};
                                p.inner_op = NEG, p.ia = m->a, p.inner_slot = 0;
                                out.push_back(p);
                            }
                        if (has(n.a, FMA, f1))   // -(A B + C) -> (-A) B + (-C)
                            for (auto* m : f1) {
                                Pending p{cls, FMA, -2, m->b, -2, 0};
                                p.inner_op = NEG, p.ia = m->a, p.inner_slot = 0;
                                p.inner2_op = NEG, p.ja = m->c, p.inner2_slot = 2;
                                out.push_back(p);
                            }
                        if (has(n.a, ADD, f1))   // -(A + B) -> (-A) - B
                            for (auto* m : f1) {
                                Pending p{cls, SUB, -2, m->b, -1, 0};
                                p.inner_op = NEG, p.ia = m->a, p.inner_slot = 0;
                                out.push_back(p);
                            }
                        if (has(n.a, SUB, f1))   // -(A - B) -> B - A
                            for (auto* m : f1) out.push_back({cls, SUB, m->b, m->a, -1, 0});
                        if (has(n.a, NEG, f1))   // -(-A) -> A
                            for (auto* m : f1) unions.push_back(cls), unions.push_back(m->a);
                    }
                    break;
            }
        }
    }

    // F_COLLECT: like-term collection over the current cheapest program. `best` is the e-node
    // extraction picks per class under positive operation costs, so following it never cycles
    // (an e-class may hold x + 0 = x after folding). For every maximal sum (a class whose best
    // node is an ADD or SUB and that no best ADD/SUB/NEG node uses), flatten it through best
    // ADD/SUB/NEG nodes into signed terms coefficient * leaf (a leaf whose best node is
    // MUL(constant, x) has that coefficient, else 1), add up the coefficients of equal leaves
    // (only where the sum is exact), drop zero terms, group the leaves by equal coefficient and
    // add  sum_g c_g * (sum of the leaves of g)  to the class, groups and leaves in order of first
    // appearance. Only sums where terms merged are rewritten. Returns the classes rewritten.
    int collect(const std::vector<std::vector<int>>& cn, const std::vector<int>& best, size_t node_limit) {
        const int nc = g.nclasses;
        auto bnode = [&](int cls) -> const Node* {
            const int b = best[g.find(cls)];
            return b >= 0 ? &g.nodes[b] : nullptr;
        };
        std::vector<char> inner(nc, 0);
        for (int c = 0; c < nc; ++c) {
            if (g.find(c) != c) continue;
            const Node* n = bnode(c);
            if (n && (n->op == ADD || n->op == SUB || n->op == NEG)) {
                inner[g.find(n->a)] = 1;
                if (n->op != NEG) inner[g.find(n->b)] = 1;
            }
        }
        std::vector<int> roots;
        for (int c = 0; c < nc; ++c) {
            if (g.find(c) != c || inner[c]) continue;
            const Node* n = bnode(c);
            if (n && (n->op == ADD || n->op == SUB)) roots.push_back(c);
        }
        int changed = 0;
        for (int root : roots) {
            if (g.nodes.size() >= node_limit) break;
            std::vector<std::pair<int, double>> terms;   // (leaf class, signed coefficient)
            std::vector<std::pair<int, double>> stack{{root, 1.0}};
            bool overflow = false;
            while (!stack.empty() && !overflow) {
                auto [cls, sign] = stack.back();
                stack.pop_back();
                const Node* sn = bnode(cls);
                if (sn && (sn->op == ADD || sn->op == SUB || sn->op == NEG)) {
                    if (terms.size() + stack.size() > 96) {
                        overflow = true;
                        break;
                    }
                    if (sn->op == NEG) {
                        stack.push_back({sn->a, -sign});
                    } else {   // right child first so the left subtree's terms come first
                        stack.push_back({sn->b, sn->op == SUB ? -sign : sign});
                        stack.push_back({sn->a, sign});
                    }
                    continue;
                }
                double v;
                if (g.const_value(cn, cls, &v) && v == 0.0) continue;   // x + 0
                double coef = sign;
                int leaf = g.find(cls);
                if (sn && sn->op == MUL) {
                    double cv;
                    if (g.const_value(cn, sn->a, &cv) && !g.const_value(cn, sn->b, &v))
                        coef = sign * cv, leaf = g.find(sn->b);
                    else if (g.const_value(cn, sn->b, &cv) && !g.const_value(cn, sn->a, &v))
                        coef = sign * cv, leaf = g.find(sn->a);
                }
                terms.push_back({leaf, coef});
            }
            if (overflow || terms.size() < 2) continue;
            // equal leaves: add their coefficients where the sum is exact
            std::vector<std::pair<int, double>> merged;
            for (auto& t : terms) {
                bool done = false;
                for (auto& m : merged) {
                    double r;
                    if (m.first == t.first && exact_add(m.second, t.second, &r)) {
                        m.second = r;
                        done = true;
                        break;
                    }
                }
                if (!done) merged.push_back(t);
            }
            merged.erase(std::remove_if(merged.begin(), merged.end(), [](const std::pair<int, double>& t) {
                             return t.second == 0.0;
                         }),
                         merged.end());
            if (merged.empty()) continue;
            std::vector<std::pair<double, std::vector<int>>> groups;   // by signed coefficient
            for (auto& t : merged) {
                bool done = false;
                for (auto& gr : groups)
                    if (gr.first == t.second) {
                        gr.second.push_back(t.first);
                        done = true;
                        break;
                    }
                if (!done) groups.push_back({t.second, {t.first}});
            }
            if (groups.size() == terms.size()) continue;   // nothing merged
            int total = -1;
            for (auto& gr : groups) {
                int S = gr.second[0];
                for (size_t q = 1; q < gr.second.size(); ++q) S = g.add(ADD, S, gr.second[q]);
                const double c = gr.first, ac = std::fabs(c);
                const int term = ac == 1.0 ? S : g.add(MUL, g.cnst(ac), S);
                if (total < 0)
                    total = c > 0 ? term : g.add(NEG, term);
                else
                    total = g.add(c > 0 ? ADD : SUB, total, term);
            }
            if (g.merge(total, root)) ++changed;
        }
        return changed;
    }

    // Apply matches; returns the number of new nodes or merges.
    int apply(std::vector<Pending>& ps, std::vector<int>& unions, size_t node_limit) {
        int changes = 0;
        for (auto& p : ps) {
            if (g.nodes.size() >= node_limit) break;
            int args[3] = {p.a, p.b, p.c};
            if (p.inner_slot >= 0) {
                int inner;
                if (p.inner_op == NEG || p.inner_op == RCP)
                    inner = g.add(p.inner_op, p.ia);
                else
                    inner = g.add(p.inner_op, p.ia, p.ib);
                args[p.inner_slot] = inner;
            }
            if (p.inner2_slot >= 0)
                args[p.inner2_slot] = p.inner2_op == NEG ? g.add(NEG, p.ja) : g.add(p.inner2_op, p.ja, p.jb);
            const size_t before = g.nodes.size();
            const int nc = g.add(p.op, args[0], args[1], args[2], p.payload);
            if (g.merge(nc, p.cls) || g.nodes.size() != before) ++changes;
        }
        for (size_t i = 0; i + 1 < unions.size(); i += 2)
            if (g.merge(unions[i], unions[i + 1])) ++changes;
        return changes;
    }
};

// ------------------------------------------------------------------ extraction

struct Extracted {
    std::vector<int> best;  // best node per canonical class (-1 if none)
};

static const double kPaperCost[NOPS] = {0.0, 1.0, 100.0, 10.0, 10.0, 10.0, 100.0, 10.0, 10.0, 100.0, 100.0};

inline Extracted extract(EGraph& g, const double* opcost) {
    auto cn = g.class_nodes();
    const int nc = g.nclasses;
    std::vector<double> cost(nc, INFINITY);
    Extracted ex;
    ex.best.assign(nc, -1);
    for (int pass = 0; pass < 200; ++pass) {
        bool changed = false;
        for (int c = 0; c < nc; ++c) {
            if (g.find(c) != c) continue;
            for (int ni : cn[c]) {
                const Node& n = g.nodes[ni];
                double s = opcost[n.op];
                const int ar = arity(n.op);
                if (ar > 0) s += cost[g.find(n.a)];
                if (ar > 1) s += cost[g.find(n.b)];
                if (ar > 2) s += cost[g.find(n.c)];
                if (s < cost[c] - 1e-9) {
                    cost[c] = s;
                    ex.best[c] = ni;
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    return ex;
}

// Extraction for a loop body, used by the march scope:
//  - an operation whose operands are all constants or parameters (an e-class computable from
//    them alone) is computed once, outside the loop over points, and costs nothing;
//  - the cost of a program is its DAG cost: every class it uses is paid once, however many
//    operations share it, which is the quantity the paper's extraction minimises (Sec. IV-B,
//    solved there as an ILP). Here a greedy tree-cost extraction is improved by local search:
//    each class of the program tries each of its e-nodes, and a change is kept when the DAG
//    cost of the whole program drops (and the choice stays acyclic), until no change helps or
//    `rounds` passes are done.
inline Extracted extract_dag(EGraph& g, const double* opcost, const std::vector<int>& outs, int rounds = 4) {
    auto cn = g.class_nodes();
    const int nc = g.nclasses;
    // classes computable from constants and parameters alone
    std::vector<char> inv(nc, 0);
    for (bool changed = true; changed;) {
        changed = false;
        for (int c = 0; c < nc; ++c) {
            if (g.find(c) != c || inv[c]) continue;
            for (int ni : cn[c]) {
                const Node& n = g.nodes[ni];
                const int ar = arity(n.op);
                bool all = n.op == CONST || n.op == PARAM || ar > 0;
                if (n.op == LOAD || n.op == FLUX) all = false;
                if (ar > 0) all = all && inv[g.find(n.a)];
                if (ar > 1) all = all && inv[g.find(n.b)];
                if (ar > 2) all = all && inv[g.find(n.c)];
                if (all) {
                    inv[c] = 1;
                    changed = true;
                    break;
                }
            }
        }
    }
    auto own = [&](const Node& n) -> double {
        const int ar = arity(n.op);
        if (ar == 0) return n.op == CONST ? 0.0 : opcost[n.op];
        bool all = inv[g.find(n.a)] && (ar < 2 || inv[g.find(n.b)]) && (ar < 3 || inv[g.find(n.c)]);
        return all ? 0.0 : opcost[n.op];
    };
    // greedy tree-cost start
    std::vector<double> cost(nc, INFINITY);
    Extracted ex;
    ex.best.assign(nc, -1);
    for (int pass = 0; pass < 200; ++pass) {
        bool changed = false;
        for (int c = 0; c < nc; ++c) {
            if (g.find(c) != c) continue;
            for (int ni : cn[c]) {
                const Node& n = g.nodes[ni];
                double sc = own(n);
                const int ar = arity(n.op);
                if (ar > 0) sc += cost[g.find(n.a)];
                if (ar > 1) sc += cost[g.find(n.b)];
                if (ar > 2) sc += cost[g.find(n.c)];
                if (sc < cost[c] - 1e-9) {
                    cost[c] = sc;
                    ex.best[c] = ni;
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    for (int r : outs)
        if (ex.best[g.find(r)] < 0) return ex;
    // DAG cost of the program under the current choice; -1 if the choice is cyclic
    std::vector<int> mark(nc, 0);
    int stamp = 0;
    auto dag_cost = [&](double* out) -> bool {
        ++stamp;
        double total = 0.0;
        std::vector<std::pair<int, int>> st;   // iterative DFS; mark -stamp = on the path
        for (int r : outs) {
            const int root = g.find(r);
            if (mark[root] == stamp) continue;
            st.push_back({root, 0});
            mark[root] = -stamp;   // on path
            while (!st.empty()) {
                auto& top = st.back();
                const int c = top.first;
                const Node& n = g.nodes[ex.best[c]];
                const int ar = arity(n.op);
                if (top.second < ar) {
                    const int ch = g.find(top.second == 0 ? n.a : top.second == 1 ? n.b : n.c);
                    ++top.second;
                    if (mark[ch] == -stamp) return false;   // cycle
                    if (mark[ch] != stamp) {
                        if (ex.best[ch] < 0) return false;
                        mark[ch] = -stamp;
                        st.push_back({ch, 0});
                    }
                    continue;
                }
                mark[c] = stamp;
                total += own(n);
                st.pop_back();
            }
        }
        *out = total;
        return true;
    };
    double cur;
    if (!dag_cost(&cur)) return ex;
    for (int round = 0; round < rounds; ++round) {
        bool improved = false;
        // the classes the program uses now
        std::vector<int> used;
        for (int c = 0; c < nc; ++c)
            if (g.find(c) == c && mark[c] == stamp) used.push_back(c);
        for (int c : used) {
            const int keep = ex.best[c];
            for (int ni : cn[c]) {
                if (ni == keep || ni == ex.best[c]) continue;
                const int prev = ex.best[c];
                ex.best[c] = ni;
                double t;
                if (dag_cost(&t) && t < cur - 1e-9) {
                    cur = t;
                    improved = true;
                } else {
                    ex.best[c] = prev;
                }
            }
        }
        dag_cost(&cur);   // refresh the marks of the used classes
        if (!improved) break;
    }
    return ex;
}

// Runs the families in the given order, iteration after iteration, until nothing changes, the
// iteration limit is reached or the e-graph holds node_limit e-nodes. Returns the iterations run.
inline int saturate(EGraph& g, const std::vector<int>& fams, int max_iters, size_t node_limit) {
    Rewriter rw(g);
    int iters = 0;
    for (iters = 0; iters < max_iters && g.nodes.size() < node_limit; ++iters) {
        int changes = 0;
        for (int f : fams) {
            auto cn = g.class_nodes();
            if (f == F_COLLECT) {
                changes += rw.collect(cn, extract(g, kPaperCost).best, node_limit);
            } else {
                std::vector<Pending> ps;
                std::vector<int> unions;
                rw.match(f, cn, ps, unions);
                changes += rw.apply(ps, unions, node_limit);
            }
            g.rebuild();
            if (g.nodes.size() >= node_limit) break;
        }
        if (changes == 0) break;
    }
    return iters;
}

}  // namespace rw
}  // namespace acs
