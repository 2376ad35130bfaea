// Host rewriter, cross-iteration scope: saturated march kernels of the RHS body.
//
// The paper rewrites each loop iteration's body on its own (Sec. IV-A). Sharing across
// neighbouring iterations, which the saturated RHS kernel does by hand, amounts to one more
// common subexpression: the flux of a point, F_d(q), is the same expression in every statement
// that differences it. Splitting the as-written RHS at that subexpression gives two bodies,
// each rewritten by equality saturation (Table I rules and the rule families of egraph.h) and
// extracted under the paper's cost model (Sec. V-B) on its own e-graph:
//   flux body     at one point q: rho, m, E -> the 12 values F_d,s(q), d = x, y, z, s = 1..4
//                 (F_d,0 = m_d needs no arithmetic), exactly as the as-written statements
//                 write them (v_d = m_d / rho, KE = 0.5 |m|^2 / rho, P = (gamma - 1)(E - KE));
//   combine body  at one point p, per component c: R_c = -sum_d (F_d,c(p+e_d) - F_d,c(p-e_d))
//                 (1/(2h_d)) - eps sum_d D4_d U_c(p), with the neighbour fluxes F_d,c(p+-e_d)
//                 as leaves (FLUX nodes; for c = 0 they are the momentum loads themselves).
// Composing the two extracted programs gives back the as-written value up to rounding (every
// rule is an identity over the reals). The variant is then emitted into the march kernel of
// march_template.h: the flux program becomes `vflux`, evaluated once per point and shared
// with the six neighbours (x/y through shared memory, z through a register queue), the combine
// program `vcombine`. A variant also draws how it is lowered to GB300 instructions (FMA forms
// with constants staged in registers or plain operations, the refined reciprocal or IEEE
// division for rcp nodes, loads first or at first use), its tile, its plane staging (TMA or
// cp.async) and its schedule (balanced or z-chunks).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "acs_internal.cuh"
#include "egraph.h"
#include "march_template.h"

namespace acs {
namespace rw {
namespace {

struct FluxBody {
    int out[3][4];   // F_d,s for s = 1..4
};

// The flux statements of the as-written RHS at one point (loads of point 0).
FluxBody build_flux_body(EGraph& g) {
    auto ld = [&](int c) { return g.add(LOAD, -1, -1, -1, (int64_t)c * 13); };
    const int gamma = g.add(PARAM, -1, -1, -1, P_GAMMA);
    const int rho = ld(0), m[3] = {ld(1), ld(2), ld(3)}, E = ld(4);
    FluxBody fb;
    for (int d = 0; d < 3; ++d) {
        const int v = g.add(DIV, m[d], rho);
        const int sq = g.add(ADD, g.add(ADD, g.add(MUL, m[0], m[0]), g.add(MUL, m[1], m[1])), g.add(MUL, m[2], m[2]));
        const int KE = g.add(DIV, g.add(MUL, g.cnst(0.5), sq), rho);
        const int P = g.add(MUL, g.add(SUB, gamma, g.cnst(1.0)), g.add(SUB, E, KE));
        for (int s = 1; s <= 4; ++s) {
            int f;
            if (s == 4) {
                f = g.add(MUL, g.add(ADD, E, P), v);
            } else {
                f = g.add(MUL, m[s - 1], v);
                if (s - 1 == d) f = g.add(ADD, f, P);
            }
            fb.out[d][s - 1] = f;
        }
    }
    return fb;
}

int pt13(int d, int sgn, int dist) { return (dist == 1 ? 1 : 7) + 2 * d + (sgn > 0 ? 0 : 1); }

// The five statements with the neighbour fluxes as leaves.
struct CombineBody {
    int root[5];
};
CombineBody build_combine_body(EGraph& g) {
    auto ld = [&](int c, int t) { return g.add(LOAD, -1, -1, -1, (int64_t)c * 13 + t); };
    auto prm = [&](int k) { return g.add(PARAM, -1, -1, -1, k); };
    const int eps = prm(P_EPS);
    const int hinv[3] = {prm(P_HX), prm(P_HY), prm(P_HZ)};
    auto F = [&](int s, int d, int side) {   // side 0: p + e_d, 1: p - e_d
        if (s == 0) return ld(d + 1, pt13(d, side ? -1 : +1, 1));
        return g.add(FLUX, -1, -1, -1, (int64_t)d * 8 + (s - 1) * 2 + side);
    };
    CombineBody b;
    for (int s = 0; s < 5; ++s) {
        int fl = g.cnst(0.0);
        for (int d = 0; d < 3; ++d) {
            const int diff = g.add(SUB, F(s, d, 0), F(s, d, 1));
            fl = g.add(ADD, fl, g.add(MUL, diff, hinv[d]));
        }
        int diss = g.cnst(0.0);
        for (int d = 0; d < 3; ++d) {
            int t4 = g.add(SUB, ld(s, pt13(d, -1, 2)), g.add(MUL, g.cnst(4.0), ld(s, pt13(d, -1, 1))));
            t4 = g.add(ADD, t4, g.add(MUL, g.cnst(6.0), ld(s, 0)));
            t4 = g.add(SUB, t4, g.add(MUL, g.cnst(4.0), ld(s, pt13(d, +1, 1))));
            t4 = g.add(ADD, t4, ld(s, pt13(d, +1, 2)));
            diss = g.add(ADD, diss, t4);
        }
        b.root[s] = g.add(SUB, g.add(NEG, fl), g.add(MUL, eps, diss));
    }
    return b;
}

std::string hexd(double v) {
    char buf[64];
    snprintf(buf, sizeof(buf), "%a", v);
    return buf;
}

void offsets13(int t, int* di, int* dj, int* dk) {
    *di = *dj = *dk = 0;
    if (t == 0) return;
    const int q = t <= 6 ? t - 1 : t - 7, d = q >> 1, mag = (t <= 6 ? 1 : 2) * ((q & 1) ? -1 : 1);
    (d == 0 ? *di : d == 1 ? *dj : *dk) = mag;
}

// Lowering choices of one variant.
struct Lowering {
    bool pipe;      // add/sub/mul as FMAs with staged 1, -1, -0; constants staged in registers
    bool rcpfast;   // rcp nodes as the refined hardware reciprocal (else IEEE 1.0 / x)
    bool bulk;      // combine: every leaf read before the arithmetic
};

// One extracted program in emission order, with its counts.
struct Emitted {
    std::vector<int> order;          // canonical classes
    std::vector<int> out_after;      // outputs stored after order[out_after[o] - 1]
    std::vector<char> invariant;     // per class: depends only on constants and parameters
    int cnt[NOPS] = {0};             // per-point operations (invariant ones excluded)
    int n_rcp_fast = 0;
    int max_live = 0;
    double cost = 0.0;               // the paper's cost of the DAG, shared classes once
};

Emitted order_program(EGraph& g, const Extracted& ex, const std::vector<int>& outs, bool bulk, const Lowering& lw) {
    Emitted e;
    const int nc = g.nclasses;
    std::vector<char> emitted(nc, 0);
    e.invariant.assign(nc, 0);
    auto emit_from = [&](int root) {
        std::vector<std::pair<int, int>> st{{g.find(root), 0}};
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
            e.order.push_back(c);
            st.pop_back();
        }
    };
    if (bulk) {
        std::vector<std::pair<int64_t, int>> leaves;   // (op, payload) order: loads, then fluxes
        std::vector<char> seen(nc, 0);
        std::vector<int> stack;
        for (int r : outs) stack.push_back(g.find(r));
        while (!stack.empty()) {
            const int c = stack.back();
            stack.pop_back();
            if (seen[c]) continue;
            seen[c] = 1;
            const Node& n = g.nodes[ex.best[c]];
            if (n.op == LOAD || n.op == FLUX) leaves.push_back({(int64_t)n.op * 1000 + n.payload, c});
            const int ar = arity(n.op);
            if (ar > 0) stack.push_back(g.find(n.a));
            if (ar > 1) stack.push_back(g.find(n.b));
            if (ar > 2) stack.push_back(g.find(n.c));
        }
        std::sort(leaves.begin(), leaves.end());
        for (auto& l : leaves) {
            emitted[l.second] = 1;
            e.order.push_back(l.second);
        }
    }
    for (int r : outs) {
        emit_from(r);
        e.out_after.push_back((int)e.order.size());
    }
    std::vector<int> last_use(nc, -1);
    for (size_t i = 0; i < e.order.size(); ++i) {
        const int c = e.order[i];
        const Node& n = g.nodes[ex.best[c]];
        const int ar = arity(n.op);
        bool inv = n.op == CONST || n.op == PARAM;
        if (ar > 0) {
            inv = true;
            const int ch[3] = {g.find(n.a), ar > 1 ? g.find(n.b) : -1, ar > 2 ? g.find(n.c) : -1};
            for (int q = 0; q < ar; ++q) {
                inv = inv && e.invariant[ch[q]];
                last_use[ch[q]] = std::max(last_use[ch[q]], (int)i);
            }
        }
        e.invariant[c] = inv;
        e.cost += kPaperCost[n.op];
        if (!inv) {
            e.cnt[n.op]++;
            if (n.op == RCP && lw.rcpfast) e.n_rcp_fast++;
        }
    }
    for (size_t o = 0; o < outs.size(); ++o) {
        const int c = g.find(outs[o]);
        last_use[c] = std::max(last_use[c], e.out_after[o]);
    }
    std::vector<int> delta(e.order.size() + 2, 0);
    for (size_t i = 0; i < e.order.size(); ++i) {
        if (e.invariant[e.order[i]]) continue;
        delta[i] += 1;
        delta[std::max(last_use[e.order[i]], (int)i) + 1] -= 1;
    }
    int live = 0;
    for (size_t i = 0; i < e.order.size(); ++i) {
        live += delta[i];
        e.max_live = std::max(e.max_live, live);
    }
    return e;
}

// Staged constant table: q[0..4] parameters, q[5..7] = 1, -1, -0, then the DAG constants.
constexpr int kNqMax = 64;
struct ConstTable {
    std::vector<double> vals;   // q[8...]
    int index(double v) {
        for (size_t i = 0; i < vals.size(); ++i)
            if (std::memcmp(&vals[i], &v, 8) == 0) return 8 + (int)i;
        if (8 + (int)vals.size() >= kNqMax) return -1;   // table full: a literal
        vals.push_back(v);
        return 7 + (int)vals.size();
    }
};

// C expression of extracted class c (operands as temporaries t<class>).
std::string expr_of(EGraph& g, const Node& n, const Lowering& lw, ConstTable& ct, bool flux_body) {
    auto tn = [&](int c) { return "t" + std::to_string(g.find(c)); };
    const int ar = arity(n.op);
    const std::string A = ar > 0 ? tn(n.a) : "", B = ar > 1 ? tn(n.b) : "", C = ar > 2 ? tn(n.c) : "";
    char buf[256];
    switch (n.op) {
        case CONST: {
            double v;
            std::memcpy(&v, &n.payload, 8);
            const int q = lw.pipe ? ct.index(v) : -1;
            return q >= 0 ? "k.q[" + std::to_string(q) + "]" : "(" + hexd(v) + ")";
        }
        case PARAM: return "k.q[" + std::to_string(n.payload) + "]";
        case LOAD: {
            const int comp = (int)(n.payload / 13), t = (int)(n.payload % 13);
            if (flux_body) return "u" + std::to_string(comp);
            int di, dj, dk;
            offsets13(t, &di, &dj, &dk);
            static const char* slots[5] = {"sm2", "sm1", "s0", "sp1", "sp2"};
            snprintf(buf, sizeof(buf), "%s[%d * PLANE + own + (%d) + (%d) * PX]", slots[dk + 2], comp, di, dj);
            return buf;
        }
        case FLUX: {
            const int d = (int)(n.payload / 8), c1 = (int)(n.payload % 8) / 2, side = (int)(n.payload % 2);
            if (d == 0)
                snprintf(buf, sizeof(buf), "Fxr[%d * ACS_BY * (ACS_BX + 2) + %d]", c1, side ? 0 : 2);
            else if (d == 1)
                snprintf(buf, sizeof(buf), "Fyr[%d * (ACS_BY + 2) * ACS_BX + %s]", c1, side ? "0" : "2 * ACS_BX");
            else
                snprintf(buf, sizeof(buf), "%s[%d]", side ? "fzm" : "fzp", c1);
            return buf;
        }
        case ADD: return lw.pipe ? "fma(" + A + ", k.q[5], " + B + ")" : A + " + " + B;
        case SUB: return lw.pipe ? "fma(" + B + ", k.q[6], " + A + ")" : A + " - " + B;
        case MUL: return lw.pipe ? "fma(" + A + ", " + B + ", k.q[7])" : A + " * " + B;
        case DIV: return A + " / " + B;
        case FMA: return "fma(" + A + ", " + B + ", " + C + ")";
        case NEG: return "-" + A;
        case RCP: return lw.rcpfast ? "rcp_fast(" + A + ", k.q[5])" : "1.0 / " + A;
    }
    return "0";
}

void dag_lines(EGraph& g, const Extracted& ex, const Emitted& e, std::string& dag) {
    char buf[160];
    for (int c : e.order) {
        const Node& n = g.nodes[ex.best[c]];
        const int ar = arity(n.op);
        snprintf(buf, sizeof(buf), "%d %s %d %d %d %lld\n", c, kOpName[n.op], ar > 0 ? g.find(n.a) : -1,
                 ar > 1 ? g.find(n.b) : -1, ar > 2 ? g.find(n.c) : -1, (long long)n.payload);
        dag += buf;
    }
}

struct TileChoice {
    int bx, by;
};
const TileChoice kTiles[6] = {{16, 16}, {32, 8}, {16, 8}, {32, 4}, {32, 16}, {64, 4}};

}  // namespace
}  // namespace rw

acs_status variant_generate_march(unsigned long long seed, int index, char* src, size_t src_len, char* dag,
                                  size_t dag_len, acs_variant_info* info) {
    using namespace rw;
    EGraph gf, gc;
    const FluxBody fb = build_flux_body(gf);
    gf.rebuild();
    const CombineBody cb = build_combine_body(gc);
    gc.rebuild();
    Rng rng(seed ^ (0x6C8E9CF570932BD5ULL * (unsigned long long)(index + 1)));
    int iters = 0;
    Lowering lw{true, true, false};
    TileChoice tile = kTiles[0];
    int flags = ACS_TILE_TMA | ACS_TILE_BALANCED;
    double opcost[NOPS];
    for (int k = 0; k < NOPS; ++k) opcost[k] = kPaperCost[k];
    if (index > 0) {
        auto draw_fams = [&]() {
            std::vector<int> fams;
            for (int f = 0; f < NFAM; ++f) {
                const double pon = (f == F_FMA || f == F_FOLD || f == F_DIV) ? 0.8
                                   : f == F_COLLECT                          ? 0.7
                                   : (f == F_EXPAND || f == F_NEGPUSH)       ? 0.5
                                                                             : 0.55;
                if (rng.uniform() < pon) fams.push_back(f);
            }
            for (int k = (int)fams.size() - 1; k > 0; --k) std::swap(fams[k], fams[rng.below(k + 1)]);
            return fams;
        };
        const std::vector<int> ff = draw_fams();
        const int fi = 1 + rng.below(10);
        const size_t fl = 2000 + (size_t)rng.below(8001);
        iters = saturate(gf, ff, fi, fl);
        const std::vector<int> fc = draw_fams();
        const int ci = 1 + rng.below(10);
        const size_t cl = 2000 + (size_t)rng.below(8001);
        iters = std::max(iters, saturate(gc, fc, ci, cl));
        for (int k = CONST + 1; k < NOPS; ++k) opcost[k] *= 0.6 + 0.8 * rng.uniform();
        // Lowering and launch priors lean to the choices the built-in kernel measured fast (FMA
        // forms with staged constants, the refined reciprocal, TMA staging, the balanced schedule,
        // 16 x 16 and 32 x 8 tiles), so that the space holds enough near-best variants to rank.
        lw.pipe = rng.uniform() < 0.75;
        lw.rcpfast = rng.uniform() < 0.9;
        lw.bulk = rng.uniform() < 0.5;
        const double u = rng.uniform();
        tile = kTiles[u < 0.3 ? 0 : u < 0.55 ? 1 : u < 0.7 ? 2 : u < 0.8 ? 3 : u < 0.9 ? 4 : 5];
        flags = (rng.uniform() < 0.8 ? ACS_TILE_TMA : 0) | (rng.uniform() < 0.7 ? ACS_TILE_BALANCED : 0);
    }
    std::vector<int> fouts, couts;
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 4; ++s) fouts.push_back(fb.out[d][s]);
    for (int s = 0; s < 5; ++s) couts.push_back(cb.root[s]);
    const Extracted exf = extract_dag(gf, opcost, fouts);
    const Extracted exc = extract_dag(gc, opcost, couts);
    for (int r : fouts)
        if (exf.best[gf.find(r)] < 0) return fail(ACS_ERR_INVALID, "flux extraction failed");
    for (int r : couts)
        if (exc.best[gc.find(r)] < 0) return fail(ACS_ERR_INVALID, "combine extraction failed");
    const Emitted ef = order_program(gf, exf, fouts, false, lw);
    const Emitted ec = order_program(gc, exc, couts, lw.bulk, lw);

    // ---- source
    ConstTable ct;
    std::string body_f, body_c;
    for (size_t i = 0, o = 0; i < ef.order.size(); ++i) {
        const int c = ef.order[i];
        body_f += "    const double t" + std::to_string(c) + " = " + expr_of(gf, gf.nodes[exf.best[c]], lw, ct, true) +
                  ";\n";
        while (o < fouts.size() && ef.out_after[o] == (int)i + 1) {
            static const char* arr[3] = {"fx", "fy", "fz"};
            body_f += "    " + std::string(arr[o / 4]) + "[" + std::to_string(o % 4) + "] = t" +
                      std::to_string(gf.find(fouts[o])) + ";\n";
            ++o;
        }
    }
    for (size_t i = 0, o = 0; i < ec.order.size(); ++i) {
        const int c = ec.order[i];
        body_c += "    const double t" + std::to_string(c) + " = " + expr_of(gc, gc.nodes[exc.best[c]], lw, ct, false) +
                  ";\n";
        while (o < couts.size() && ec.out_after[o] == (int)i + 1) {
            body_c += "    Rp[" + std::to_string(o) + " * osc] = t" + std::to_string(gc.find(couts[o])) + ";\n";
            ++o;
        }
    }
    const int nq = 8 + (int)ct.vals.size();
    const int nt = tile.bx * tile.by;
    char hdr[512];
    snprintf(hdr, sizeof(hdr),
             "// generated by the acs host rewriter: cross-iteration saturated march kernel\n"
             "#define ACS_BX %d\n#define ACS_BY %d\n#define ACS_TMA %d\n#define ACS_BALANCED %d\n"
             "#define ACS_NQ %d\n#define ACS_NQ_PAD %d\n#define ACS_MINB %d\n",
             tile.bx, tile.by, (flags & ACS_TILE_TMA) ? 1 : 0, (flags & ACS_TILE_BALANCED) ? 1 : 0, nq, kNqMax,
             nt <= 256 ? 2 : 1);
    std::string s = hdr;
    s += kMarchPrelude;
    s += "struct VK { double q[ACS_NQ]; };\n";
    s += "__device__ __forceinline__ void vk_stage(double* Cs, const VP& vp) {\n"
         "    Cs[0] = vp.gamma; Cs[1] = vp.eps; Cs[2] = vp.hx; Cs[3] = vp.hy; Cs[4] = vp.hz;\n"
         "    Cs[5] = 1.0; Cs[6] = -1.0; Cs[7] = -0.0;\n";
    for (size_t i = 0; i < ct.vals.size(); ++i) s += "    Cs[" + std::to_string(8 + i) + "] = " + hexd(ct.vals[i]) + ";\n";
    s += "}\n";
    s += "__device__ __forceinline__ void vflux(double u0, double u1, double u2, double u3, double u4, const VK& k,\n"
         "                                      double fx[4], double fy[4], double fz[4]) {\n";
    s += body_f + "}\n";
    s += "__device__ __forceinline__ void vcombine(const double* __restrict__ sm2, const double* __restrict__ sm1,\n"
         "    const double* __restrict__ s0, const double* __restrict__ sp1, const double* __restrict__ sp2, int own,\n"
         "    const double* __restrict__ Fxr, const double* __restrict__ Fyr, const double fzm[4], const double fzp[4],\n"
         "    double* __restrict__ Rp, i64 osc, const VK& k) {\n";
    s += body_c + "}\n";
    s += kMarchKernel;

    // ---- DAG text
    std::string d = "flux\n";
    dag_lines(gf, exf, ef, d);
    char buf[96];
    for (size_t o = 0; o < fouts.size(); ++o) {
        snprintf(buf, sizeof(buf), "F %zu %zu %d\n", o / 4, o % 4 + 1, gf.find(fouts[o]));
        d += buf;
    }
    d += "combine\n";
    dag_lines(gc, exc, ec, d);
    for (size_t o = 0; o < couts.size(); ++o) {
        snprintf(buf, sizeof(buf), "R %zu %d\n", o, gc.find(couts[o]));
        d += buf;
    }

    // ---- features (per interior point)
    float f[ACS_VARIANT_NFEAT];
    std::fill(f, f + ACS_VARIANT_NFEAT, 0.f);
    auto both = [&](int op) { return ef.cnt[op] + ec.cnt[op]; };
    const int n_arith_f = ef.cnt[ADD] + ef.cnt[SUB] + ef.cnt[MUL] + ef.cnt[FMA];
    const int n_arith_c = ec.cnt[ADD] + ec.cnt[SUB] + ec.cnt[MUL] + ec.cnt[FMA];
    const int slow_f = ef.cnt[DIV] + (ef.cnt[RCP] - ef.n_rcp_fast);
    const int slow_c = ec.cnt[DIV] + (ec.cnt[RCP] - ec.n_rcp_fast);
    const double flux_ops = n_arith_f + 9.0 * slow_f + 4.0 * ef.n_rcp_fast;
    const double comb_ops = n_arith_c + 9.0 * slow_c + 4.0 * ec.n_rcp_fast;
    // the flux ring: 2 (BX + BY) threads in whole warps, out of BX BY / 32 warps
    const double ring_warps = std::ceil(2.0 * tile.bx / 32.0) + std::ceil(2.0 * tile.by / 32.0);
    const double ring_frac = ring_warps / (nt / 32.0);
    f[0] = (float)(ef.cost + ec.cost);
    f[1] = (float)(both(ADD) + both(SUB));
    f[2] = (float)both(MUL);
    f[3] = (float)both(FMA);
    f[4] = (float)(both(DIV) + both(RCP) - ef.n_rcp_fast - ec.n_rcp_fast);
    f[5] = (float)both(NEG);
    f[6] = (float)(ec.cnt[LOAD] + ec.cnt[FLUX] + 5);
    f[7] = (float)ec.cnt[LOAD];
    f[8] = (float)ec.cnt[FLUX];
    f[9] = (float)(ef.order.size() + ec.order.size());
    f[10] = (float)std::max(ef.max_live, ec.max_live);
    f[11] = lw.bulk ? 1.f : 0.f;
    f[12] = lw.pipe ? 1.f : 0.f;
    f[13] = (float)tile.bx;
    f[14] = 0.f;   // registers, filled after compilation
    f[15] = (float)(flux_ops * (1.0 + ring_frac) + comb_ops);
    f[16] = (float)tile.by;
    f[17] = (flags & ACS_TILE_TMA) ? 1.f : 0.f;
    f[18] = (flags & ACS_TILE_BALANCED) ? 1.f : 0.f;
    f[19] = (float)(ef.n_rcp_fast + ec.n_rcp_fast);
    if (info) {
        std::memcpy(info->feats, f, sizeof(f));
        info->cost = ef.cost + ec.cost;
        int ncls = 0;
        for (int c = 0; c < gf.nclasses; ++c) ncls += gf.find(c) == c;
        for (int c = 0; c < gc.nclasses; ++c) ncls += gc.find(c) == c;
        info->enodes = (int)(gf.nodes.size() + gc.nodes.size());
        info->eclasses = ncls;
        info->iterations = iters;
        info->scope = ACS_SCOPE_MARCH;
        info->block_x = tile.bx;
        info->block_y = tile.by;
        info->flags = flags;
        info->src_bytes = (long long)s.size() + 1;
        info->dag_bytes = (long long)d.size() + 1;
    }
    if (src) {
        if (s.size() + 1 > src_len) return fail(ACS_ERR_INVALID, "source buffer too small (%zu needed)", s.size() + 1);
        std::memcpy(src, s.c_str(), s.size() + 1);
    }
    if (dag) {
        if (d.size() + 1 > dag_len) return fail(ACS_ERR_INVALID, "dag buffer too small (%zu needed)", d.size() + 1);
        std::memcpy(dag, d.c_str(), d.size() + 1);
    }
    return ACS_OK;
}

}  // namespace acs
