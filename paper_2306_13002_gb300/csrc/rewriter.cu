// Host-side rewriter of the RHS loop body: e-graph, equality saturation, extraction, codegen.
//
// This follows the paper's pipeline (Sec. IV-VI) on the one body this library evaluates:
//  1. The as-written body (the five statements of rhs_plain.cu, loads as leaves) is added to
//     an e-graph; identical subexpressions share an e-class from the start (hash-consing).
//  2. Saturation applies rewrite rules to every e-node until nothing changes or a limit is
//     hit: 10,000 e-nodes, 10 iterations by default (Sec. VII-A). Rule families: the Table I
//     rules (FMA1-3, COMM-ADD/MUL, ASSOC-ADD1/2, ASSOC-MUL1/2), constant folding, and the
//     families the paper can express but leaves off to keep e-graphs small (Sec. V-A):
//     division (a/b -> a * rcp(b), moving a product out of a quotient), distributivity and
//     subtraction/negation. A variant draws which families are on, their order within an
//     iteration, the iteration and node limits, from its own counter-based random stream,
//     so different variants stop in different parts of the space ("random rule orders").
//  3. Extraction picks one e-node per e-class bottom-up under the paper's cost model
//     (Sec. V-B: constants 0, inputs 1, arithmetic 10, memory access / division 100), each
//     variant scaling the operation costs by its own random factors; the extracted program
//     is a DAG whose shared e-classes are computed once (common subexpressions).
//  4. Code generation emits one temporary per extracted e-class in first-use order or with
//     every load first (bulk load, Sec. VI-B), as a CUDA kernel compiled at run time.
// Every rule is an identity over the reals (constant folding is applied only when the
// folded double is exact), so every variant computes the as-written value up to rounding.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "acs_internal.cuh"
#include "egraph.h"

namespace acs {
namespace rw {

// ------------------------------------------------------------------ the as-written body

struct Body {
    int root[5];
};

// Point index t of the 13-point body: 0 = p, 1..6 = +-e_x,+-e_y,+-e_z, 7..12 = +-2e_d.
static int pt(int d, int sgn, int dist) { return (dist == 1 ? 1 : 7) + 2 * d + (sgn > 0 ? 0 : 1); }

Body build_as_written(EGraph& g) {
    auto ld = [&](int c, int t) { return g.add(LOAD, -1, -1, -1, (int64_t)c * 13 + t); };
    auto prm = [&](int k) { return g.add(PARAM, -1, -1, -1, k); };
    const int gamma = prm(P_GAMMA), eps = prm(P_EPS);
    const int hinv[3] = {prm(P_HX), prm(P_HY), prm(P_HZ)};
    // flux component s along axis d at neighbour point t (as written in rhs_plain.cu)
    auto flux = [&](int s, int d, int t) {
        const int rho = ld(0, t), m[3] = {ld(1, t), ld(2, t), ld(3, t)}, E = ld(4, t);
        if (s == 0) return m[d];
        const int v = g.add(DIV, m[d], rho);
        const int sq = g.add(ADD, g.add(ADD, g.add(MUL, m[0], m[0]), g.add(MUL, m[1], m[1])), g.add(MUL, m[2], m[2]));
        const int KE = g.add(DIV, g.add(MUL, g.cnst(0.5), sq), rho);
        const int P = g.add(MUL, g.add(SUB, gamma, g.cnst(1.0)), g.add(SUB, E, KE));
        if (s == 4) return g.add(MUL, g.add(ADD, E, P), v);
        int f = g.add(MUL, m[s - 1], v);
        if (s - 1 == d) f = g.add(ADD, f, P);
        return f;
    };
    Body b;
    for (int s = 0; s < 5; ++s) {
        int fl = g.cnst(0.0);
        for (int d = 0; d < 3; ++d) {
            const int diff = g.add(SUB, flux(s, d, pt(d, +1, 1)), flux(s, d, pt(d, -1, 1)));
            fl = g.add(ADD, fl, g.add(MUL, diff, hinv[d]));
        }
        int diss = g.cnst(0.0);
        for (int d = 0; d < 3; ++d) {
            int t4 = g.add(SUB, ld(s, pt(d, -1, 2)), g.add(MUL, g.cnst(4.0), ld(s, pt(d, -1, 1))));
            t4 = g.add(ADD, t4, g.add(MUL, g.cnst(6.0), ld(s, 0)));
            t4 = g.add(SUB, t4, g.add(MUL, g.cnst(4.0), ld(s, pt(d, +1, 1))));
            t4 = g.add(ADD, t4, ld(s, pt(d, +1, 2)));
            diss = g.add(ADD, diss, t4);
        }
        b.root[s] = g.add(SUB, g.add(NEG, fl), g.add(MUL, eps, diss));
    }
    return b;
}

// ------------------------------------------------------------------ codegen + features

struct Program {
    std::vector<int> order;   // canonical classes in emission order
    std::vector<int> store_after;  // store_after[s] = index in order after which R_s is stored
    std::string src, dag;
    float feats[ACS_VARIANT_NFEAT];
    double cost;
};

static std::string hexd(double v) {
    char buf[64];
    snprintf(buf, sizeof(buf), "%a", v);
    return buf;
}

static void point_offsets(int t, int* di, int* dj, int* dk) {
    *di = *dj = *dk = 0;
    if (t == 0) return;
    const int q = t <= 6 ? t - 1 : t - 7, d = q >> 1, mag = (t <= 6 ? 1 : 2) * ((q & 1) ? -1 : 1);
    (d == 0 ? *di : d == 1 ? *dj : *dk) = mag;
}

Program codegen(EGraph& g, const Extracted& ex, const Body& body, bool bulk, bool pipe, int bx) {
    Program pr;
    const int nc = g.nclasses;
    std::vector<char> emitted(nc, 0);
    std::vector<int> order;
    // DFS post-order from a root (iterative to bound stack depth)
    auto emit_from = [&](int root) {
        std::vector<std::pair<int, int>> st;
        st.push_back({g.find(root), 0});
        while (!st.empty()) {
            auto& top = st.back();
            const int c = top.first;
            if (emitted[c]) {
                st.pop_back();
                continue;
            }
            const Node& n = g.nodes[ex.best[c]];
            const int ar = arity(n.op);
            if (top.second < ar) {
                const int ch = g.find(top.second == 0 ? n.a : top.second == 1 ? n.b : n.c);
                ++top.second;
                if (!emitted[ch]) st.push_back({ch, 0});
                continue;
            }
            emitted[c] = 1;
            order.push_back(c);
            st.pop_back();
        }
    };
    if (bulk) {
        // every load first, sorted by static index (component, point)
        std::vector<std::pair<int64_t, int>> loads;
        std::vector<char> seen(nc, 0);
        for (int s = 0; s < 5; ++s) {
            std::vector<int> stack{g.find(body.root[s])};
            while (!stack.empty()) {
                const int c = stack.back();
                stack.pop_back();
                if (seen[c]) continue;
                seen[c] = 1;
                const Node& n = g.nodes[ex.best[c]];
                if (n.op == LOAD) loads.push_back({n.payload, c});
                const int ar = arity(n.op);
                if (ar > 0) stack.push_back(g.find(n.a));
                if (ar > 1) stack.push_back(g.find(n.b));
                if (ar > 2) stack.push_back(g.find(n.c));
            }
        }
        std::sort(loads.begin(), loads.end());
        for (auto& l : loads) {
            emitted[l.second] = 1;
            order.push_back(l.second);
        }
    }
    std::vector<int> store_after(5);
    for (int s = 0; s < 5; ++s) {
        emit_from(body.root[s]);
        store_after[s] = (int)order.size();
    }
    // features
    int cnt[NOPS] = {0};
    int nload_x = 0, nload_yz = 0;
    double cost = 0.0;
    std::vector<int> pos(nc, -1), last_use(nc, -1);
    for (size_t i = 0; i < order.size(); ++i) pos[order[i]] = (int)i;
    for (size_t i = 0; i < order.size(); ++i) {
        const Node& n = g.nodes[ex.best[order[i]]];
        cnt[n.op]++;
        cost += kPaperCost[n.op];
        if (n.op == LOAD) {
            const int t = (int)(n.payload % 13);
            int di, dj, dk;
            point_offsets(t, &di, &dj, &dk);
            if (dj == 0 && dk == 0)
                ++nload_x;
            else
                ++nload_yz;
        }
        const int ar = arity(n.op);
        const int ch[3] = {ar > 0 ? g.find(n.a) : -1, ar > 1 ? g.find(n.b) : -1, ar > 2 ? g.find(n.c) : -1};
        for (int k = 0; k < ar; ++k) last_use[ch[k]] = std::max(last_use[ch[k]], (int)i);
    }
    for (int s = 0; s < 5; ++s) last_use[g.find(body.root[s])] = std::max(last_use[g.find(body.root[s])], store_after[s]);
    // register-pressure estimate: most temporaries live at once in emission order
    std::vector<int> delta(order.size() + 2, 0);
    for (size_t i = 0; i < order.size(); ++i) {
        const Node& n = g.nodes[ex.best[order[i]]];
        if (n.op == CONST || n.op == PARAM) continue;
        const int lu = std::max(last_use[order[i]], (int)i);
        delta[i] += 1;
        delta[lu + 1] -= 1;
    }
    int live = 0, max_live = 0;
    for (size_t i = 0; i < order.size(); ++i) {
        live += delta[i];
        max_live = std::max(max_live, live);
    }
    const int n_arith = cnt[ADD] + cnt[SUB] + cnt[MUL] + cnt[FMA];
    float* f = pr.feats;
    std::fill(f, f + ACS_VARIANT_NFEAT, 0.f);
    f[0] = (float)cost;
    f[1] = (float)(cnt[ADD] + cnt[SUB]);
    f[2] = (float)cnt[MUL];
    f[3] = (float)cnt[FMA];
    f[4] = (float)(cnt[DIV] + cnt[RCP]);
    f[5] = (float)cnt[NEG];
    f[6] = (float)cnt[LOAD];
    f[7] = (float)nload_x;
    f[8] = (float)nload_yz;
    f[9] = (float)order.size();
    f[10] = (float)max_live;
    f[11] = bulk ? 1.f : 0.f;
    f[12] = pipe ? 1.f : 0.f;
    f[13] = (float)bx;
    f[14] = 0.f;  // registers, filled after compilation
    f[15] = (float)(n_arith + 9 * (cnt[DIV] + cnt[RCP]));
    f[16] = (float)(256 / bx);   // block_y; tma, balanced, n_rcp_fast stay 0
    pr.cost = cost;

    // CUDA source
    std::string s;
    s.reserve(order.size() * 64 + 2048);
    s += "// generated by the acs host rewriter\n";
    s += "struct VArgs { int nx, ny, nz, halo; long long isy, isz, isc, osy, osz, osc; double q[8]; };\n";
    char buf[512];
    snprintf(buf, sizeof(buf),
             "extern \"C\" __global__ void __launch_bounds__(256) acs_variant(const double* U, double* R, VArgs a) {\n"
             "  const int i = blockIdx.x * %d + threadIdx.x %% %d;\n"
             "  const int j = blockIdx.y * %d + threadIdx.x / %d;\n"
             "  if (i >= a.nx || j >= a.ny) return;\n"
             "  for (int k = blockIdx.z; k < a.nz; k += gridDim.z) {\n"
             "  const long long p = (long long)(k + a.halo) * a.isz + (long long)(j + a.halo) * a.isy + (i + a.halo);\n"
             "  double* Rp = R + (long long)k * a.osz + (long long)j * a.osy + i;\n",
             bx, bx, 256 / bx, bx);
    s += buf;
    auto tn = [&](int c) { return "t" + std::to_string(c); };
    size_t next_store = 0;
    std::string dag;
    for (size_t i = 0; i < order.size(); ++i) {
        const int c = order[i];
        const Node& n = g.nodes[ex.best[c]];
        const int ar = arity(n.op);
        std::string A = ar > 0 ? tn(g.find(n.a)) : "", B = ar > 1 ? tn(g.find(n.b)) : "", C = ar > 2 ? tn(g.find(n.c)) : "";
        std::string e;
        switch (n.op) {
            case CONST: {
                double v;
                std::memcpy(&v, &n.payload, 8);
                e = hexd(v);
                break;
            }
            case PARAM: e = "a.q[" + std::to_string(n.payload) + "]"; break;
            case LOAD: {
                const int comp = (int)(n.payload / 13), t = (int)(n.payload % 13);
                int di, dj, dk;
                point_offsets(t, &di, &dj, &dk);
                snprintf(buf, sizeof(buf), "U[%d * a.isc + p + (%d) + (%d) * a.isy + (%d) * a.isz]", comp, di, dj, dk);
                e = buf;
                break;
            }
            case ADD: e = pipe ? "fma(" + A + ", a.q[5], " + B + ")" : A + " + " + B; break;
            case SUB: e = pipe ? "fma(" + B + ", a.q[6], " + A + ")" : A + " - " + B; break;
            case MUL: e = pipe ? "fma(" + A + ", " + B + ", a.q[7])" : A + " * " + B; break;
            case DIV: e = A + " / " + B; break;
            case FMA: e = "fma(" + A + ", " + B + ", " + C + ")"; break;
            case NEG: e = "-" + A; break;
            case RCP: e = "1.0 / " + A; break;
        }
        s += "  const double " + tn(c) + " = " + e + ";\n";
        snprintf(buf, sizeof(buf), "%d %s %d %d %d %lld\n", c, kOpName[n.op], ar > 0 ? g.find(n.a) : -1,
                 ar > 1 ? g.find(n.b) : -1, ar > 2 ? g.find(n.c) : -1, (long long)n.payload);
        dag += buf;
        while (next_store < 5 && store_after[next_store] == (int)i + 1) {
            s += "  Rp[" + std::to_string(next_store) + " * a.osc] = " + tn(g.find(body.root[next_store])) + ";\n";
            snprintf(buf, sizeof(buf), "R %zu %d\n", next_store, g.find(body.root[next_store]));
            dag += buf;
            ++next_store;
        }
    }
    while (next_store < 5) {
        s += "  Rp[" + std::to_string(next_store) + " * a.osc] = " + tn(g.find(body.root[next_store])) + ";\n";
        snprintf(buf, sizeof(buf), "R %zu %d\n", next_store, g.find(body.root[next_store]));
        dag += buf;
        ++next_store;
    }
    s += "  }\n}\n";
    pr.src = s;
    pr.dag = dag;
    pr.order = order;
    pr.store_after = store_after;
    return pr;
}

}  // namespace rw

static const char* kFeatureNames[ACS_VARIANT_NFEAT] = {
    "paper_cost", "n_add", "n_mul", "n_fma", "n_div", "n_neg", "n_load", "n_load_x", "n_load_yz", "n_nodes",
    "max_live", "bulk", "pipe", "block_x", "regs", "dp_ops_est", "block_y", "tma", "balanced", "n_rcp_fast"};

const char* variant_feature_name(int i) { return (i >= 0 && i < ACS_VARIANT_NFEAT) ? kFeatureNames[i] : ""; }

acs_status variant_generate(unsigned long long seed, int index, char* src, size_t src_len, char* dag, size_t dag_len,
                            acs_variant_info* info) {
    using namespace rw;
    EGraph g;
    Body body = build_as_written(g);
    g.rebuild();
    Rng rng(seed ^ (0xA5A5A5A5ULL * (unsigned long long)(index + 1)));
    int iters = 0;
    bool bulk = false, pipe = false;
    int bx = 32;
    double opcost[NOPS];
    for (int k = 0; k < NOPS; ++k) opcost[k] = kPaperCost[k];
    if (index > 0) {
        // variant-specific rule families, order, limits and cost perturbation
        std::vector<int> fams;
        for (int f = 0; f < NFAM_PAPER; ++f) {
            const double pon = (f == F_FMA || f == F_FOLD) ? 0.8 : 0.55;
            if (rng.uniform() < pon) fams.push_back(f);
        }
        for (int k = (int)fams.size() - 1; k > 0; --k) std::swap(fams[k], fams[rng.below(k + 1)]);
        const int max_iters = 1 + rng.below(10);
        const size_t node_limit = 2000 + (size_t)rng.below(8001);
        iters = saturate(g, fams, max_iters, node_limit);
        for (int k = CONST + 1; k <= RCP; ++k) opcost[k] *= 0.6 + 0.8 * rng.uniform();
        bulk = rng.uniform() < 0.5;
        pipe = rng.uniform() < 0.5;
        static const int bxs[3] = {32, 64, 128};
        bx = bxs[rng.below(3)];
    }
    Extracted ex = extract(g, opcost);
    for (int s = 0; s < 5; ++s)
        if (ex.best[g.find(body.root[s])] < 0) return fail(ACS_ERR_INVALID, "extraction failed for statement %d", s);
    Program pr = codegen(g, ex, body, bulk, pipe, bx);
    if (info) {
        std::memcpy(info->feats, pr.feats, sizeof(pr.feats));
        info->cost = pr.cost;
        info->enodes = (int)g.nodes.size();
        int ncls = 0;
        for (int c = 0; c < g.nclasses; ++c) ncls += g.find(c) == c;
        info->eclasses = ncls;
        info->iterations = iters;
        info->scope = ACS_SCOPE_ITERATION;
        info->block_x = bx;
        info->block_y = 256 / bx;
        info->flags = 0;
        info->src_bytes = (long long)pr.src.size() + 1;
        info->dag_bytes = (long long)pr.dag.size() + 1;
    }
    if (src) {
        if (pr.src.size() + 1 > src_len) return fail(ACS_ERR_INVALID, "source buffer too small (%zu needed)", pr.src.size() + 1);
        std::memcpy(src, pr.src.c_str(), pr.src.size() + 1);
    }
    if (dag) {
        if (pr.dag.size() + 1 > dag_len) return fail(ACS_ERR_INVALID, "dag buffer too small (%zu needed)", pr.dag.size() + 1);
        std::memcpy(dag, pr.dag.c_str(), pr.dag.size() + 1);
    }
    return ACS_OK;
}

}  // namespace acs
