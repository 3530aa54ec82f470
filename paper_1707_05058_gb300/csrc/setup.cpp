// Host data preprocessing of Algorithms 1-3 (arXiv 1707.05058): aggregate
// pattern (Section 2.1), chordal extension and maximal cliques (Section 7.1.1),
// entry selectors H_k and D = sum_k H_k^T H_k (Section 4), the cached
// inverses of A D^-1 A^T (Eq. ADMMprimalFatorization) and of
// I + A (I + D/2)^-1 A^T (Eq. HSDEFactorizationFinal), and zeta_hat
// (Proposition 2).  Runs once per problem, on the CPU; not on the hot path.
//
// Canonical rules (fixed so that results are reproducible bit for bit):
//  * chordality: maximum cardinality search, ties to the smallest vertex; the
//    reverse visiting order is tested as a perfect elimination order (PEO).
//  * non-chordal patterns: exact minimum-degree elimination game, ties to the
//    smallest vertex; eliminating v joins its remaining neighbours.
//  * maximal cliques: K_v = {v} U later-neighbours(v) is kept unless some u
//    with parent(u) = v has |later(u)| = |later(v)| + 1 (parent = first later
//    neighbour); cliques sorted ascending, list sorted lexicographically.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <iterator>
#include <map>
#include <memory>
#include <new>
#include <queue>
#include <set>
#include <tuple>
#include <thread>
#include <utility>

#include "cdsdp_internal.h"

namespace cdsdp_impl {
namespace {

// Run body(t) for t = 0 .. T-1 on T host threads (T = hardware threads, at
// most `cap`); plain loop when one thread is enough.
constexpr int kSetupThreads = 16;  // cap on threads of the triplet loops
constexpr size_t kBitsetMaxOrder = 32768;  // bit-matrix elimination graph up to n^2/8 = 128 MB
constexpr size_t kBucketBitsBytes = 256u << 20;  // cap on the bit-set buckets of the cardinality search

// Barrier for the threads of one parallel_threads call (all of them run at
// once); spins briefly, then yields.
class SpinBarrier {
  public:
    explicit SpinBarrier(int n) : n_(n) {}
    void wait() {
        const int g = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
            return;
        }
        for (int spins = 0; gen_.load(std::memory_order_acquire) == g; ++spins)
            if (spins > 256) std::this_thread::yield();
    }

  private:
    std::atomic<int> count_{0}, gen_{0};
    const int n_;
};

template <typename F>
void parallel_threads(int cap, F&& body) {
    int T = (int)std::thread::hardware_concurrency();
    T = std::max(1, std::min(T, cap));
    if (T == 1) { body(0, 1); return; }
    std::vector<std::thread> th;
    th.reserve(T - 1);
    for (int t = 1; t < T; ++t) th.emplace_back([&body, t, T]() { body(t, T); });
    body(0, T);
    for (auto& x : th) x.join();
}

// Dense Cholesky (lower, row-major, in place) followed by the explicit
// inverse inv = L^-T L^-1: the columns of L^-1 by forward substitution, then
// inv_ij = <column i, column j>, both in parallel over columns; every inner
// loop runs along contiguous memory.  Returns false on a non-positive pivot.
bool spd_inverse(std::vector<double>& a, int m, std::vector<double>& inv, int threads) {
    double maxdiag = 0.0;
    for (int i = 0; i < m; ++i) maxdiag = std::max(maxdiag, std::fabs(a[(size_t)i * m + i]));
    // Cholesky by columns; the rows below the pivot are shared out, row i to
    // thread i mod T, which also owns the pivot of column i; one barrier per
    // column.  Every element sees the same operations in the same order for
    // any T.
    const int TC = m >= 256 ? std::max(1, std::min(threads, (int)std::thread::hardware_concurrency())) : 1;
    SpinBarrier bar(TC);
    std::atomic<int> bad(0);
    parallel_threads(TC, [&](int t, int T) {
        for (int j = 0; j < m; ++j) {
            double* rj = &a[(size_t)j * m];
            if (j % T == t) {
                double d = rj[j];
                for (int k = 0; k < j; ++k) d -= rj[k] * rj[k];
                if (!(d > 1e-14 * maxdiag)) bad.store(1, std::memory_order_relaxed);
                else rj[j] = std::sqrt(d);
            }
            if (T > 1) bar.wait();
            if (bad.load(std::memory_order_relaxed)) return;
            const double ljj = rj[j];
            for (int i = j + 1 + ((t - j - 1) % T + T) % T; i < m; i += T) {
                double* ri = &a[(size_t)i * m];
                double s = ri[j];
                for (int k = 0; k < j; ++k) s -= ri[k] * rj[k];
                ri[j] = s / ljj;
            }
        }
    });
    if (bad) return false;
    // xt row j = column j of L^-1 (entries j..m-1): L x = e_j
    std::vector<double> xt((size_t)m * m, 0.0);
    const int cap = m >= 128 ? threads : 1;
    parallel_threads(cap, [&](int t, int T) {
        for (int j = t; j < m; j += T) {
            double* x = &xt[(size_t)j * m];
            for (int i = j; i < m; ++i) {
                const double* li = &a[(size_t)i * m];
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) s -= li[k] * x[k];
                x[i] = s / li[i];
            }
        }
    });
    inv.assign((size_t)m * m, 0.0);
    parallel_threads(cap, [&](int t, int T) {
        for (int i = t; i < m; i += T) {
            const double* xi = &xt[(size_t)i * m];
            for (int j = 0; j <= i; ++j) {
                const double* xj = &xt[(size_t)j * m];
                double s = 0.0;
                for (int k = i; k < m; ++k) s += xi[k] * xj[k];  // k >= max(i, j) = i
                inv[(size_t)i * m + j] = s;
                inv[(size_t)j * m + i] = s;
            }
        }
    });
    return true;
}

// Clique merging (an option, not in the paper): coarser cliques of a further
// chordal extension when they cut the projection work sum |C|^3.  The rule is
// fixed so that it can be restated independently:
//  1. clique tree = maximum-weight spanning forest of the clique intersection
//     graph (weight |C_i ^ C_j| > 0), Kruskal over edges (i < j) taken in the
//     order (weight descending, i ascending, j ascending);
//  2. repeatedly take the tree edge with the largest gain
//     |C_i|^3 + |C_j|^3 - |C_i u C_j|^3 (ties: smaller min(i, j), then smaller
//     max(i, j)) while that gain is positive; node min(i, j) becomes
//     C_i u C_j and inherits the other node's tree edges;
//  3. the surviving cliques, each ascending, sorted lexicographically.
// Merging two cliques adjacent in a clique tree keeps the graph chordal and
// the contracted tree a clique tree.
std::vector<std::vector<int>> merge_cliques(const std::vector<std::vector<int>>& cl, int n) {
    const int p = (int)cl.size();
    std::vector<std::vector<int>> members(n);
    for (int k = 0; k < p; ++k)
        for (int v : cl[k]) members[v].push_back(k);
    std::map<std::pair<int, int>, int> inter;
    for (int v = 0; v < n; ++v) {
        const auto& ks = members[v];
        for (size_t a = 0; a < ks.size(); ++a)
            for (size_t c = a + 1; c < ks.size(); ++c) ++inter[{ks[a], ks[c]}];
    }
    struct E { int w, i, j; };
    std::vector<E> edges;
    edges.reserve(inter.size());
    for (const auto& kv : inter) edges.push_back({kv.second, kv.first.first, kv.first.second});
    std::sort(edges.begin(), edges.end(), [](const E& x, const E& y) {
        if (x.w != y.w) return x.w > y.w;
        if (x.i != y.i) return x.i < y.i;
        return x.j < y.j;
    });
    std::vector<int> uf(p);
    for (int k = 0; k < p; ++k) uf[k] = k;
    auto find = [&](int x) {
        while (uf[x] != x) x = uf[x] = uf[uf[x]];
        return x;
    };
    std::vector<std::set<int>> adj(p);
    for (const E& e : edges) {
        const int ri = find(e.i), rj = find(e.j);
        if (ri == rj) continue;
        uf[ri] = rj;
        adj[e.i].insert(e.j);
        adj[e.j].insert(e.i);
    }
    std::vector<std::vector<int>> sets(cl);
    std::vector<char> alive(p, 1);
    auto cube = [](long long x) { return x * x * x; };
    auto gain = [&](int i, int j) {
        std::vector<int> u;
        std::set_union(sets[i].begin(), sets[i].end(), sets[j].begin(), sets[j].end(), std::back_inserter(u));
        return cube((long long)sets[i].size()) + cube((long long)sets[j].size()) - cube((long long)u.size());
    };
    // max-heap on (gain, -lo, -hi): the largest gain, then the smallest ids
    using H = std::tuple<long long, int, int>;
    std::priority_queue<H> heap;
    auto push = [&](int i, int j) {
        const int lo = std::min(i, j), hi = std::max(i, j);
        heap.push(H{gain(lo, hi), -lo, -hi});
    };
    for (int i = 0; i < p; ++i)
        for (int j : adj[i])
            if (i < j) push(i, j);
    while (!heap.empty()) {
        const auto [g, nlo, nhi] = heap.top();
        heap.pop();
        const int lo = -nlo, hi = -nhi;
        if (!alive[lo] || !alive[hi] || !adj[lo].count(hi)) continue;
        if (g != gain(lo, hi)) continue;  // stale: a fresh entry for this edge is in the heap
        if (g <= 0) break;
        std::vector<int> u;
        std::set_union(sets[lo].begin(), sets[lo].end(), sets[hi].begin(), sets[hi].end(), std::back_inserter(u));
        sets[lo] = std::move(u);
        alive[hi] = 0;
        adj[lo].erase(hi);
        for (int c : adj[hi]) {
            if (c == lo) continue;
            adj[c].erase(hi);
            adj[c].insert(lo);
            adj[lo].insert(c);
        }
        adj[hi].clear();
        for (int c : adj[lo]) push(lo, c);
    }
    std::vector<std::vector<int>> out;
    for (int k = 0; k < p; ++k)
        if (alive[k]) out.push_back(sets[k]);
    std::sort(out.begin(), out.end());
    return out;
}

int entry_of(const HostProblem& hp, int i, int j) {  // i >= j
    const int* beg = hp.prow.data() + hp.colptr[j];
    const int* end = hp.prow.data() + hp.colptr[j + 1];
    const int* it = std::lower_bound(beg, end, i);
    if (it == end || *it != i) return -1;
    return (int)(it - hp.prow.data());
}

}  // namespace

// Cached inverse of A W diag(d)^-1 A^T (+ I for the HSDE system, d = 1 + D/2),
// block diagonal over the independent components (Eqs.
// ADMMprimalFatorization, HSDEFactorizationFinal).
int build_factor(const HostProblem& hp, bool hsde, std::vector<double>& inv) {
    const int NE = (int)hp.prow.size(), m = hp.m;
    auto wgt = [&](int e) { return hp.prow[e] == hp.pcol[e] ? 1.0 : 2.0; };
    if (hp.diag_factor) {
        inv.assign(m, hsde ? 1.0 : 0.0);
        for (int e = 0; e < NE; ++e)
            for (int q = hp.at_ptr[e]; q < hp.at_ptr[e + 1]; ++q) {
                const double dd = hsde ? 1.0 + 0.5 * hp.D[e] : hp.D[e];
                inv[hp.at_col[q]] += wgt(e) * hp.at_val[q] * hp.at_val[q] / dd;
            }
        for (int i = 0; i < m; ++i) {
            if (!(inv[i] > 0.0)) return CDSDP_ERR_RANK;
            inv[i] = 1.0 / inv[i];
        }
        return CDSDP_SOLVED;
    }
    inv.assign((size_t)hp.factor_size, 0.0);
    std::vector<std::vector<double>> blocks(hp.ncomp);
    for (int c = 0; c < hp.ncomp; ++c) {
        const int mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
        blocks[c].assign((size_t)mc * mc, 0.0);
        for (int i = 0; hsde && i < mc; ++i) blocks[c][(size_t)i * mc + i] = 1.0;
    }
    // lower triangle of each block (the constraints of an A^T row are in
    // ascending order, hence so are their positions in the block), then mirror
    // (every element gets its terms in entry order whatever the threading:
    // one component -> threads own the block rows r with r mod T = t and each
    // scans every entry; several -> threads take whole components)
    auto accumulate = [&](int e, std::vector<int>& lr, int th, int T) {
        const int c = hp.comp_of_entry[e];
        const int mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
        double* S = blocks[c].data();
        const double f = wgt(e) / (hsde ? 1.0 + 0.5 * hp.D[e] : hp.D[e]);
        const int q0 = hp.at_ptr[e], nq = hp.at_ptr[e + 1] - q0;
        lr.resize(nq);
        for (int u = 0; u < nq; ++u) lr[u] = hp.lrow[hp.at_col[q0 + u]];
        const double* av = &hp.at_val[q0];
        for (int u = 0; u < nq; ++u) {
            if (lr[u] % T != th) continue;
            const double v1 = f * av[u];
            double* row = S + (size_t)lr[u] * mc;
            for (int w = 0; w <= u; ++w) row[lr[w]] += v1 * av[w];
        }
    };
    const int TS = hp.at_ptr[NE] >= (1 << 16) ? kSetupThreads : 1;
    if (hp.ncomp == 1) {
        parallel_threads(TS, [&](int th, int T) {
            std::vector<int> lr;
            for (int e = 0; e < NE; ++e) accumulate(e, lr, th, T);
        });
    } else {
        std::vector<int> eptr(hp.ncomp + 1, 0), eidx(NE);
        for (int e = 0; e < NE; ++e) ++eptr[hp.comp_of_entry[e] + 1];
        for (int c = 0; c < hp.ncomp; ++c) eptr[c + 1] += eptr[c];
        {
            std::vector<int> fill(eptr.begin(), eptr.end() - 1);
            for (int e = 0; e < NE; ++e) eidx[fill[hp.comp_of_entry[e]]++] = e;
        }
        std::atomic<int> next(0);
        parallel_threads(TS, [&](int, int) {
            std::vector<int> lr;
            for (int c = next++; c < hp.ncomp; c = next++)
                for (int q = eptr[c]; q < eptr[c + 1]; ++q) accumulate(eidx[q], lr, 0, 1);
        });
    }
    for (int c = 0; c < hp.ncomp; ++c) {
        const int mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
        double* S = blocks[c].data();
        for (int i = 0; i < mc; ++i)
            for (int j = 0; j < i; ++j) S[(size_t)j * mc + i] = S[(size_t)i * mc + j];
    }
    // one component: threads inside the inverse; several: one component per thread
    std::atomic<int> bad(0);
    if (hp.ncomp == 1) {
        std::vector<double> bi;
        if (!spd_inverse(blocks[0], hp.m, bi, 16)) return CDSDP_ERR_RANK;
        std::copy(bi.begin(), bi.end(), inv.begin());
    } else {
        std::atomic<int> next(0);
        parallel_threads(16, [&](int, int) {
            for (int c = next++; c < hp.ncomp; c = next++) {
                const int mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
                std::vector<double> bi;
                if (!spd_inverse(blocks[c], mc, bi, 1)) { bad = 1; continue; }
                std::copy(bi.begin(), bi.end(), inv.begin() + hp.minv_off[c]);
            }
        });
    }
    return bad ? CDSDP_ERR_RANK : CDSDP_SOLVED;
}

int build_hsde_constants(HostProblem& hp) {
    if (hp.hsde_ready) return CDSDP_SOLVED;
    const int NE = (int)hp.prow.size(), m = hp.m;
    auto wgt = [&](int e) { return hp.prow[e] == hp.pcol[e] ? 1.0 : 2.0; };
    int st = build_factor(hp, true, hp.kinv);
    if (st != CDSDP_SOLVED) return st;
    // ---- HSDE: zeta_hat from one inner solve with nu = zeta = (c, 0, -b, 0)
    {
        auto kinv_apply = [&](const std::vector<double>& r, std::vector<double>& out) {
            out.assign(m, 0.0);
            if (hp.diag_factor) { for (int i = 0; i < m; ++i) out[i] = hp.kinv[i] * r[i]; return; }
            for (int i = 0; i < m; ++i) {
                const int c = hp.comp_of_row[i], mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
                const double* row = hp.kinv.data() + hp.minv_off[c] + (size_t)hp.lrow[i] * mc;
                double s = 0.0;
                for (int j = 0; j < mc; ++j) s += row[j] * r[hp.crow_idx[hp.crow_ptr[c] + j]];
                out[i] = s;
            }
        };
        auto A_w = [&](const std::vector<double>& x, std::vector<double>& out) {  // A W x
            out.assign(m, 0.0);
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int q = hp.a_ptr[i]; q < hp.a_ptr[i + 1]; ++q) s += hp.a_val[q] * wgt(hp.a_col[q]) * x[hp.a_col[q]];
                out[i] = s;
            }
        };
        auto A_T = [&](const std::vector<double>& y, std::vector<double>& out) {
            out.assign(NE, 0.0);
            for (int e = 0; e < NE; ++e) {
                double s = 0.0;
                for (int q = hp.at_ptr[e]; q < hp.at_ptr[e + 1]; ++q) s += hp.at_val[q] * y[hp.at_col[q]];
                out[e] = s;
            }
        };
        A_T(hp.b, hp.atb);
        std::vector<double> pe(NE), r, hh, athh, s11(NE), as11;
        for (int e = 0; e < NE; ++e) pe[e] = (hp.c[e] - hp.atb[e]) / (1.0 + 0.5 * hp.D[e]);
        A_w(pe, r);
        kinv_apply(r, hh);
        A_T(hh, athh);
        for (int e = 0; e < NE; ++e) s11[e] = pe[e] - athh[e] / (1.0 + 0.5 * hp.D[e]);
        A_w(s11, as11);
        std::vector<double> s21(m);
        for (int i = 0; i < m; ++i) s21[i] = -hp.b[i] - as11[i];
        double zMz = 0.0;
        for (int e = 0; e < NE; ++e) zMz += wgt(e) * hp.c[e] * s11[e];
        for (int i = 0; i < m; ++i) zMz -= hp.b[i] * s21[i];
        double denom = 1.0 + zMz;
        hp.zhat_x.resize(NE);
        hp.zhat_y.resize(m);
        for (int e = 0; e < NE; ++e) hp.zhat_x[e] = s11[e] / denom;
        for (int i = 0; i < m; ++i) hp.zhat_y[i] = s21[i] / denom;
        hp.zeta_dot_zhat = zMz / denom;
        A_w(hp.zhat_x, hp.a_zhat_x);
        // one embedding per component: M is block diagonal over the components,
        // so M^-1 zeta restricted to component c is M_c^-1 zeta_c (s11, s21 above),
        // normalised by that component's own 1 + zeta_c^T M_c^-1 zeta_c
        std::vector<double> zmz(hp.ncomp, 0.0);
        for (int e = 0; e < NE; ++e) zmz[hp.comp_of_entry[e]] += wgt(e) * hp.c[e] * s11[e];
        for (int i = 0; i < m; ++i) zmz[hp.comp_of_row[i]] -= hp.b[i] * s21[i];
        hp.zhat_x_c.resize(NE);
        hp.zhat_y_c.resize(m);
        hp.zdz_c.resize(hp.ncomp);
        for (int e = 0; e < NE; ++e) hp.zhat_x_c[e] = s11[e] / (1.0 + zmz[hp.comp_of_entry[e]]);
        for (int i = 0; i < m; ++i) hp.zhat_y_c[i] = s21[i] / (1.0 + zmz[hp.comp_of_row[i]]);
        for (int c = 0; c < hp.ncomp; ++c) hp.zdz_c[c] = zmz[c] / (1.0 + zmz[c]);
        A_w(hp.zhat_x_c, hp.a_zhat_x_c);
    }
    hp.hsde_ready = true;
    return CDSDP_SOLVED;
}

int build_host_problem(int n, int m,
                       long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                       const double* bvec,
                       long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                       long long nnzP, const int* P_row, const int* P_col,
                       HostProblem& hp, bool cache_factor, bool merge) {
    if (n < 1 || m < 1 || nnzA < 0 || nnzC < 0 || nnzP < 0) return CDSDP_ERR_ARG;
    if (nnzA > 0 && (!A_con || !A_row || !A_col || !A_val)) return CDSDP_ERR_ARG;
    if (nnzC > 0 && (!C_row || !C_col || !C_val)) return CDSDP_ERR_ARG;
    if (nnzP > 0 && (!P_row || !P_col)) return CDSDP_ERR_ARG;
    if (!bvec) return CDSDP_ERR_ARG;
    if (nnzA > 2000000000LL || nnzC > 2000000000LL || nnzP > 2000000000LL) return CDSDP_ERR_UNSUPPORTED;
    auto bad_pair = [n](int r, int c) { return r < 0 || c < 0 || r >= n || c >= n || r < c; };
    for (long long k = 0; k < nnzA; ++k)
        if (bad_pair(A_row[k], A_col[k]) || A_con[k] < 0 || A_con[k] >= m || !std::isfinite(A_val[k]))
            return CDSDP_ERR_ARG;
    for (long long k = 0; k < nnzC; ++k)
        if (bad_pair(C_row[k], C_col[k]) || !std::isfinite(C_val[k])) return CDSDP_ERR_ARG;
    for (long long k = 0; k < nnzP; ++k)
        if (bad_pair(P_row[k], P_col[k])) return CDSDP_ERR_ARG;
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(bvec[i])) return CDSDP_ERR_ARG;

    hp = HostProblem();
    hp.n = n;
    hp.m = m;

    // ---- aggregate pattern (off-diagonal adjacency, sorted, unique): C and
    // the extra edges first, then the entries of A that are not there yet
    // (usually none: C tends to cover the pattern of the A_i)
    std::vector<std::vector<int>> adj(n);
    auto add_edge = [&](int r, int c) {
        if (r != c) { adj[r].push_back(c); adj[c].push_back(r); }
    };
    auto tidy = [&]() {
        for (auto& a : adj) {
            std::sort(a.begin(), a.end());
            a.erase(std::unique(a.begin(), a.end()), a.end());
        }
    };
    for (long long k = 0; k < nnzC; ++k) add_edge(C_row[k], C_col[k]);
    for (long long k = 0; k < nnzP; ++k) add_edge(P_row[k], P_col[k]);
    tidy();
    {
        // entries of A not yet in the pattern: threads over chunks of the
        // triplets, results concatenated in triplet order
        const int TA = nnzA >= (1 << 16) ? kSetupThreads : 1;
        std::vector<std::vector<std::pair<int, int>>> extra_t(std::max(1, TA));
        parallel_threads(TA, [&](int t, int T) {
            const long long k0 = nnzA * t / T, k1 = nnzA * (t + 1) / T;
            auto& ex = extra_t[t];
            for (long long k = k0; k < k1; ++k) {
                const int r = A_row[k], c = A_col[k];
                if (r != c && !std::binary_search(adj[r].begin(), adj[r].end(), c)) ex.push_back({r, c});
            }
        });
        bool any = false;
        for (auto& ex : extra_t) {
            for (auto& e : ex) add_edge(e.first, e.second);
            any = any || !ex.empty();
        }
        if (any) tidy();
    }
    long long nedges = 0;
    for (auto& a : adj) {
        nedges += (long long)a.size();
    }
    nedges /= 2;

    // ---- maximum cardinality search with buckets (ties: smallest vertex)
    std::vector<int> visit;
    visit.reserve(n);
    size_t maxdeg = 0;
    for (auto& a : adj) maxdeg = std::max(maxdeg, a.size());
    const size_t W0 = ((size_t)n + 63) / 64, W1 = (W0 + 63) / 64;
    if ((maxdeg + 1) * (W0 + W1) * sizeof(uint64_t) <= kBucketBitsBytes) {
        // buckets as two-level bit sets (a word per 64 vertices, a summary bit
        // per word): the smallest vertex of the top bucket by find-first-set
        std::vector<uint64_t> lv0((maxdeg + 1) * W0, 0), lv1((maxdeg + 1) * W1, 0);
        std::vector<int> cnt(maxdeg + 1, 0), weight(n, 0);
        std::vector<char> done(n, 0);
        auto ins = [&](size_t w, int v) {
            lv0[w * W0 + (v >> 6)] |= 1ULL << (v & 63);
            lv1[w * W1 + (v >> 12)] |= 1ULL << ((v >> 6) & 63);
            ++cnt[w];
        };
        auto del = [&](size_t w, int v) {
            uint64_t& x = lv0[w * W0 + (v >> 6)];
            x &= ~(1ULL << (v & 63));
            if (!x) lv1[w * W1 + (v >> 12)] &= ~(1ULL << ((v >> 6) & 63));
            --cnt[w];
        };
        auto first = [&](size_t w) {
            for (size_t i = 0; i < W1; ++i)
                if (const uint64_t sm = lv1[w * W1 + i]) {
                    const size_t j = i * 64 + (size_t)__builtin_ctzll(sm);
                    return (int)(j * 64 + (size_t)__builtin_ctzll(lv0[w * W0 + j]));
                }
            return -1;
        };
        for (int v = 0; v < n; ++v) ins(0, v);
        size_t top = 0;
        for (int step = 0; step < n; ++step) {
            while (top > 0 && cnt[top] == 0) --top;
            const int v = first(top);
            del(top, v);
            done[v] = 1;
            visit.push_back(v);
            for (int u : adj[v]) {
                if (done[u]) continue;
                del((size_t)weight[u], u);
                ++weight[u];
                ins((size_t)weight[u], u);
                if ((size_t)weight[u] > top) top = (size_t)weight[u];
            }
        }
    } else {
        std::vector<int> weight(n, 0);
        std::vector<char> done(n, 0);
        std::vector<std::set<int>> bucket(n + 1);
        for (int v = 0; v < n; ++v) bucket[0].insert(v);
        int top = 0;
        for (int step = 0; step < n; ++step) {
            while (top > 0 && bucket[top].empty()) --top;
            int v = *bucket[top].begin();
            bucket[top].erase(bucket[top].begin());
            done[v] = 1;
            visit.push_back(v);
            for (int u : adj[v]) {
                if (done[u]) continue;
                bucket[weight[u]].erase(u);
                ++weight[u];
                bucket[weight[u]].insert(u);
                if (weight[u] > top) top = weight[u];
            }
        }
    }
    std::vector<int> elim(visit.rbegin(), visit.rend());
    std::vector<int> pos(n);
    for (int k = 0; k < n; ++k) pos[elim[k]] = k;
    // later neighbours per vertex for this order
    std::vector<std::vector<int>> later(n);
    for (int v = 0; v < n; ++v)
        for (int u : adj[v])
            if (pos[u] > pos[v]) later[v].push_back(u);
    // Tarjan-Yannakakis PEO test: later(v) \ {parent} must lie in adj(parent)
    bool chordal = true;
    for (int v = 0; v < n && chordal; ++v) {
        if (later[v].empty()) continue;
        int par = later[v][0];
        for (int u : later[v]) if (pos[u] < pos[par]) par = u;
        for (int u : later[v]) {
            if (u == par) continue;
            if (!std::binary_search(adj[par].begin(), adj[par].end(), u)) { chordal = false; break; }
        }
    }
    hp.chordal = chordal;
    if (!chordal && (size_t)n <= kBitsetMaxOrder) {
        // exact minimum-degree elimination game (ties: smallest vertex) on a
        // bit-matrix elimination graph: eliminating v ORs row v into the rows
        // of its neighbours (the fill) and clears v; degrees are popcounts
        const size_t W = ((size_t)n + 63) / 64;
        std::vector<uint64_t> bits((size_t)n * W, 0);
        auto row = [&](int v) { return bits.data() + (size_t)v * W; };
        for (int v = 0; v < n; ++v)
            for (int u : adj[v]) row(v)[u >> 6] |= 1ULL << (u & 63);
        std::vector<int> deg(n);
        std::set<std::pair<int, int>> order;
        for (int v = 0; v < n; ++v) {
            deg[v] = (int)adj[v].size();
            order.insert({deg[v], v});
        }
        // thread 0 picks each pivot and keeps the degree order; the row
        // updates of the pivot's neighbours are shared out (two barriers a step)
        std::vector<int> nb, newdeg(n);
        const int TE = std::max(1, std::min(n >= 2048 ? kSetupThreads : 1, (int)std::thread::hardware_concurrency()));
        SpinBarrier bar(TE);
        parallel_threads(TE, [&](int t, int T) {
            for (int k = 0; k < n; ++k) {
                if (t == 0) {
                    const int v = order.begin()->second;
                    order.erase(order.begin());
                    elim[k] = v;
                    pos[v] = k;
                    const uint64_t* rv = row(v);
                    nb.clear();
                    for (size_t w = 0; w < W; ++w)
                        for (uint64_t x = rv[w]; x; x &= x - 1) nb.push_back((int)(w * 64 + __builtin_ctzll(x)));
                    later[v] = nb;
                }
                bar.wait();
                const int v = elim[k];
                const uint64_t* rv = row(v);
                const uint64_t vbit = 1ULL << (v & 63);
                for (size_t a = t; a < nb.size(); a += T) {
                    const int u = nb[a];
                    uint64_t* ru = row(u);
                    for (size_t w = 0; w < W; ++w) ru[w] |= rv[w];
                    ru[u >> 6] &= ~(1ULL << (u & 63));
                    ru[v >> 6] &= ~vbit;
                    int d = 0;
                    for (size_t w = 0; w < W; ++w) d += __builtin_popcountll(ru[w]);
                    newdeg[u] = d;
                }
                bar.wait();
                if (t == 0) {
                    for (int u : nb) {
                        order.erase({deg[u], u});
                        deg[u] = newdeg[u];
                        order.insert({deg[u], u});
                    }
                    std::fill(bits.begin() + (size_t)v * W, bits.begin() + (size_t)(v + 1) * W, 0ULL);
                }
            }
        });
    } else if (!chordal) {
        // exact minimum-degree elimination game (ties: smallest vertex)
        std::vector<std::set<int>> g(n);
        for (int v = 0; v < n; ++v) g[v].insert(adj[v].begin(), adj[v].end());
        std::set<std::pair<int, int>> order;
        for (int v = 0; v < n; ++v) order.insert({(int)g[v].size(), v});
        for (int k = 0; k < n; ++k) {
            int v = order.begin()->second;
            order.erase(order.begin());
            elim[k] = v;
            pos[v] = k;
            std::vector<int> nb(g[v].begin(), g[v].end());
            later[v] = nb;
            for (int u : nb) {
                order.erase({(int)g[u].size(), u});
                g[u].erase(v);
            }
            for (size_t a = 0; a < nb.size(); ++a)
                for (size_t c2 = a + 1; c2 < nb.size(); ++c2) {
                    int x = nb[a], y = nb[c2];
                    if (g[x].insert(y).second) g[y].insert(x);
                }
            for (int u : nb) order.insert({(int)g[u].size(), u});
            g[v].clear();
        }
    }
    for (auto& l : later) std::sort(l.begin(), l.end());
    hp.peo = elim;
    hp.lt_ptr.assign(n + 1, 0);
    for (int v = 0; v < n; ++v) hp.lt_ptr[v + 1] = hp.lt_ptr[v] + (int)later[v].size();
    hp.lt_idx.clear();
    hp.lt_idx.reserve(hp.lt_ptr[n]);
    for (int v = 0; v < n; ++v) hp.lt_idx.insert(hp.lt_idx.end(), later[v].begin(), later[v].end());

    // ---- maximal cliques (parent rule on the PEO)
    std::vector<char> maximal(n, 1);
    for (int u = 0; u < n; ++u) {
        if (later[u].empty()) continue;
        int par = later[u][0];
        for (int x : later[u]) if (pos[x] < pos[par]) par = x;
        if (later[u].size() == later[par].size() + 1) maximal[par] = 0;
    }
    std::vector<std::vector<int>> cliques;
    for (int v = 0; v < n; ++v) {
        if (!maximal[v]) continue;
        std::vector<int> k = later[v];
        k.push_back(v);
        std::sort(k.begin(), k.end());
        cliques.push_back(std::move(k));
    }
    std::sort(cliques.begin(), cliques.end());
    if (merge) {
        cliques = merge_cliques(cliques, n);
        hp.merged = true;
    }
    hp.cl_off.assign(1, 0);
    for (auto& k : cliques) {
        hp.cl_vert.insert(hp.cl_vert.end(), k.begin(), k.end());
        hp.cl_off.push_back((int)hp.cl_vert.size());
        hp.max_clique = std::max(hp.max_clique, (int)k.size());
    }

    // ---- extended pattern, lower, column-major
    {
        std::vector<std::vector<int>> col(n);
        long long off = 0;
        if (!merge) {
            for (int v = 0; v < n; ++v) {
                col[v].push_back(v);
                for (int u : later[v]) {
                    col[std::min(u, v)].push_back(std::max(u, v));
                    ++off;
                }
            }
        } else {  // every pair within a merged clique
            for (int v = 0; v < n; ++v) col[v].push_back(v);
            for (const auto& k : cliques)
                for (size_t bb = 0; bb < k.size(); ++bb)
                    for (size_t a = bb + 1; a < k.size(); ++a) col[k[bb]].push_back(k[a]);
            for (int v = 0; v < n; ++v) {
                std::sort(col[v].begin() + 1, col[v].end());
                col[v].erase(std::unique(col[v].begin() + 1, col[v].end()), col[v].end());
                off += (long long)col[v].size() - 1;
            }
        }
        hp.nfill = off - nedges;
        hp.colptr.assign(n + 1, 0);
        for (int j = 0; j < n; ++j) {
            std::sort(col[j].begin(), col[j].end());
            hp.colptr[j + 1] = hp.colptr[j] + (int)col[j].size();
        }
        hp.prow.reserve(hp.colptr[n]);
        hp.pcol.reserve(hp.colptr[n]);
        for (int j = 0; j < n; ++j)
            for (int i : col[j]) { hp.prow.push_back(i); hp.pcol.push_back(j); }
    }
    const int NE = (int)hp.prow.size();

    // ---- H_k (gather map), H^T (scatter map), D
    const int p = (int)cliques.size();
    hp.pk_off.assign(p + 1, 0);
    for (int k = 0; k < p; ++k) hp.pk_off[k + 1] = hp.pk_off[k] + packed_size((int)cliques[k].size());
    hp.gmap.resize(hp.pk_off[p]);
    {
        // threads take whole cliques; within a clique column the rows ascend,
        // so each search starts past the previous hit
        std::atomic<int> next(0), missing(0);
        const int TG = hp.pk_off[p] >= (1 << 16) ? kSetupThreads : 1;
        parallel_threads(TG, [&](int, int) {
            for (int k = next++; k < p; k = next++) {
                const auto& cl = cliques[k];
                const int s = (int)cl.size();
                int q = hp.pk_off[k];
                for (int bb = 0; bb < s; ++bb) {
                    const int* beg = hp.prow.data() + hp.colptr[cl[bb]];
                    const int* end = hp.prow.data() + hp.colptr[cl[bb] + 1];
                    for (int a = bb; a < s; ++a) {
                        const int* it = std::lower_bound(beg, end, cl[a]);
                        if (it == end || *it != cl[a]) {  // cannot happen for a valid extension
                            missing = 1;
                            hp.gmap[q++] = 0;
                            continue;
                        }
                        hp.gmap[q++] = (int)(it - hp.prow.data());
                        beg = it + 1;
                    }
                }
            }
        });
        if (missing) return CDSDP_ERR_ARG;
    }
    hp.sc_ptr.assign(NE + 1, 0);
    hp.sc_idx.resize(hp.gmap.size());
    const long long nq = (long long)hp.gmap.size();
    if (nq < (1 << 20)) {
        for (int e : hp.gmap) ++hp.sc_ptr[e + 1];
        for (int e = 0; e < NE; ++e) hp.sc_ptr[e + 1] += hp.sc_ptr[e];
        std::vector<int> fill(hp.sc_ptr.begin(), hp.sc_ptr.end() - 1);
        for (int q = 0; q < (int)nq; ++q) hp.sc_idx[fill[hp.gmap[q]]++] = q;
    } else {
        // threads over chunks of packed positions with atomic counters and
        // cursors, then each entry's (short) position list sorted: the same
        // ascending lists as the sequential pass
        std::unique_ptr<std::atomic<int>[]> cur(new std::atomic<int>[NE]);
        for (int e = 0; e < NE; ++e) cur[e].store(0, std::memory_order_relaxed);
        parallel_threads(kSetupThreads, [&](int t, int T) {
            const long long q0 = nq * t / T, q1 = nq * (t + 1) / T;
            for (long long q = q0; q < q1; ++q) cur[hp.gmap[q]].fetch_add(1, std::memory_order_relaxed);
        });
        for (int e = 0; e < NE; ++e) {
            hp.sc_ptr[e + 1] = hp.sc_ptr[e] + cur[e].load(std::memory_order_relaxed);
            cur[e].store(hp.sc_ptr[e], std::memory_order_relaxed);
        }
        parallel_threads(kSetupThreads, [&](int t, int T) {
            const long long q0 = nq * t / T, q1 = nq * (t + 1) / T;
            for (long long q = q0; q < q1; ++q)
                hp.sc_idx[cur[hp.gmap[q]].fetch_add(1, std::memory_order_relaxed)] = (int)q;
        });
        parallel_threads(kSetupThreads, [&](int t, int T) {
            const int e0 = (int)((long long)NE * t / T), e1 = (int)((long long)NE * (t + 1) / T);
            for (int e = e0; e < e1; ++e) std::sort(hp.sc_idx.begin() + hp.sc_ptr[e], hp.sc_idx.begin() + hp.sc_ptr[e + 1]);
        });
    }
    hp.D.resize(NE);
    for (int e = 0; e < NE; ++e) hp.D[e] = (double)(hp.sc_ptr[e + 1] - hp.sc_ptr[e]);

    // ---- c, A (CSR over entries, duplicates merged), A^T
    hp.c.assign(NE, 0.0);
    for (long long k = 0; k < nnzC; ++k) hp.c[entry_of(hp, C_row[k], C_col[k])] += C_val[k];
    {
        // bucket the triplets by constraint (triplet order kept within a row),
        // sort each row by entry, merge duplicates; threads over chunks of the
        // triplets, then over rows; the result does not depend on the thread count
        const int TA = nnzA >= (1 << 16) ? kSetupThreads : 1;
        const int T = std::max(1, std::min(TA, (int)std::thread::hardware_concurrency()));
        std::vector<long long> cnt((size_t)T * m, 0);  // per chunk, per row
        parallel_threads(T, [&](int t, int TT) {
            const long long k0 = nnzA * t / TT, k1 = nnzA * (t + 1) / TT;
            long long* ct = &cnt[(size_t)t * m];
            for (long long k = k0; k < k1; ++k) ++ct[A_con[k]];
        });
        std::vector<long long> rp(m + 1, 0);
        for (int i = 0; i < m; ++i) {
            long long o = rp[i];
            for (int t = 0; t < T; ++t) {
                const long long c = cnt[(size_t)t * m + i];
                cnt[(size_t)t * m + i] = o;  // now the chunk's first slot in row i
                o += c;
            }
            rp[i + 1] = o;
        }
        // (entry, value) records, left uninitialised: the threads touch them first
        struct Rec {
            int first;
            double second;
        };
        std::unique_ptr<Rec[]> t(new Rec[(size_t)std::max(1LL, nnzA)]);
        parallel_threads(T, [&](int th, int TT) {
            const long long k0 = nnzA * th / TT, k1 = nnzA * (th + 1) / TT;
            long long* fill = &cnt[(size_t)th * m];
            for (long long k = k0; k < k1; ++k)
                t[(size_t)fill[A_con[k]]++] = {entry_of(hp, A_row[k], A_col[k]), A_val[k]};
        });
        std::vector<int> merged(m, 0);
        parallel_threads(T, [&](int th, int TT) {
            for (int i = th; i < m; i += TT) {
                Rec* b0 = t.get() + rp[i];
                Rec* b1 = t.get() + rp[i + 1];
                std::sort(b0, b1, [](const auto& x, const auto& y) { return x.first < y.first; });
                Rec* out = b0;
                for (Rec* it = b0; it != b1; ++it) {
                    if (out != b0 && (out - 1)->first == it->first) { (out - 1)->second += it->second; continue; }
                    *out++ = *it;
                }
                merged[i] = (int)(out - b0);
            }
        });
        hp.a_ptr.assign(m + 1, 0);
        for (int i = 0; i < m; ++i) hp.a_ptr[i + 1] = hp.a_ptr[i] + merged[i];
        hp.a_col.resize(hp.a_ptr[m]);
        hp.a_val.resize(hp.a_ptr[m]);
        parallel_threads(T, [&](int th, int TT) {
            for (int i = th; i < m; i += TT)
                for (int q = 0; q < merged[i]; ++q) {
                    hp.a_col[hp.a_ptr[i] + q] = t[(size_t)rp[i] + q].first;
                    hp.a_val[hp.a_ptr[i] + q] = t[(size_t)rp[i] + q].second;
                }
        });
    }
    hp.b.assign(bvec, bvec + m);

    // ---- independent components (union-find over vertices)
    {
        std::vector<int> parent(n);
        for (int v = 0; v < n; ++v) parent[v] = v;
        auto find = [&](int v) {
            while (parent[v] != v) { parent[v] = parent[parent[v]]; v = parent[v]; }
            return v;
        };
        auto unite = [&](int a, int b2) {
            a = find(a); b2 = find(b2);
            if (a != b2) parent[std::max(a, b2)] = std::min(a, b2);
        };
        for (int e = 0; e < NE; ++e) unite(hp.prow[e], hp.pcol[e]);
        for (int i = 0; i < m; ++i)
            for (int q = hp.a_ptr[i] + 1; q < hp.a_ptr[i + 1]; ++q) unite(hp.pcol[hp.a_col[q]], hp.pcol[hp.a_col[hp.a_ptr[i]]]);
        // components numbered by their smallest vertex
        std::vector<int> id(n, -1);
        hp.ncomp = 0;
        for (int v = 0; v < n; ++v) {
            const int r = find(v);
            if (id[r] < 0) id[r] = hp.ncomp++;
        }
        auto comp = [&](int v) { return id[find(v)]; };
        hp.comp_of_vertex.resize(n);
        for (int v = 0; v < n; ++v) hp.comp_of_vertex[v] = comp(v);
        hp.comp_of_entry.resize(NE);
        for (int e = 0; e < NE; ++e) hp.comp_of_entry[e] = comp(hp.pcol[e]);
        hp.comp_of_clique.resize(p);
        for (int k = 0; k < p; ++k) hp.comp_of_clique[k] = comp(hp.cl_vert[hp.cl_off[k]]);
        hp.comp_of_row.assign(m, 0);
        for (int i = 0; i < m; ++i)
            if (hp.a_ptr[i + 1] > hp.a_ptr[i]) hp.comp_of_row[i] = hp.comp_of_entry[hp.a_col[hp.a_ptr[i]]];
        const int C = hp.ncomp;
        hp.crow_ptr.assign(C + 1, 0);
        for (int i = 0; i < m; ++i) ++hp.crow_ptr[hp.comp_of_row[i] + 1];
        for (int c = 0; c < C; ++c) hp.crow_ptr[c + 1] += hp.crow_ptr[c];
        hp.crow_idx.resize(m);
        hp.lrow.resize(m);
        {
            std::vector<int> fill(hp.crow_ptr.begin(), hp.crow_ptr.end() - 1);
            for (int i = 0; i < m; ++i) {
                const int c = hp.comp_of_row[i];
                hp.lrow[i] = fill[c] - hp.crow_ptr[c];
                hp.crow_idx[fill[c]++] = i;
            }
        }
        hp.rows_contiguous = true;
        for (int i = 0; i < m; ++i)
            if (hp.crow_idx[i] != i) hp.rows_contiguous = false;
        hp.ccl_ptr.assign(C + 1, 0);
        for (int k = 0; k < p; ++k) ++hp.ccl_ptr[hp.comp_of_clique[k] + 1];
        for (int c = 0; c < C; ++c) hp.ccl_ptr[c + 1] += hp.ccl_ptr[c];
        hp.ccl_idx.resize(p);
        {
            std::vector<int> fill(hp.ccl_ptr.begin(), hp.ccl_ptr.end() - 1);
            for (int k = 0; k < p; ++k) hp.ccl_idx[fill[hp.comp_of_clique[k]]++] = k;
        }
    }

    // ---- A^T: counting sort by entry, rows ascending within an entry
    {
        const int T = std::max(1, std::min(kSetupThreads, (int)std::thread::hardware_concurrency()));
        const int nnz = hp.a_ptr[m];
        if (hp.ncomp > 1 && nnz >= (1 << 16)) {
            // the components own disjoint rows and entries: threads take whole
            // components, each walking its rows in ascending order
            hp.at_ptr.assign(NE + 1, 0);
            std::atomic<int> next(0);
            parallel_threads(T, [&](int, int) {
                for (int c = next++; c < hp.ncomp; c = next++)
                    for (int r = hp.crow_ptr[c]; r < hp.crow_ptr[c + 1]; ++r) {
                        const int i = hp.crow_idx[r];
                        for (int q = hp.a_ptr[i]; q < hp.a_ptr[i + 1]; ++q) ++hp.at_ptr[hp.a_col[q] + 1];
                    }
            });
            for (int e = 0; e < NE; ++e) hp.at_ptr[e + 1] += hp.at_ptr[e];
            hp.at_col.resize(nnz);
            hp.at_val.resize(nnz);
            std::vector<int> fill(hp.at_ptr.begin(), hp.at_ptr.end() - 1);
            next = 0;
            parallel_threads(T, [&](int, int) {
                for (int c = next++; c < hp.ncomp; c = next++)
                    for (int r = hp.crow_ptr[c]; r < hp.crow_ptr[c + 1]; ++r) {
                        const int i = hp.crow_idx[r];
                        for (int q = hp.a_ptr[i]; q < hp.a_ptr[i + 1]; ++q) {
                            const int dst = fill[hp.a_col[q]]++;
                            hp.at_col[dst] = i;
                            hp.at_val[dst] = hp.a_val[q];
                        }
                    }
            });
        } else {
            // threads over contiguous row ranges when their per-entry counters fit
            const int TT2 = ((size_t)T * (NE + 1) * sizeof(int) <= (64u << 20) && nnz >= (1 << 16)) ? T : 1;
            std::vector<int> rb(TT2 + 1, m);  // rows of chunk t: [rb[t], rb[t+1]), about nnz / TT2 each
            rb[0] = 0;
            for (int th = 1, i = 0; th < TT2; ++th) {
                const long long target = (long long)nnz * th / TT2;
                while (i < m && hp.a_ptr[i] < target) ++i;
                rb[th] = i;
            }
            std::vector<int> ecnt((size_t)TT2 * NE, 0);
            parallel_threads(TT2, [&](int th, int) {
                int* ec = &ecnt[(size_t)th * NE];
                for (int q = hp.a_ptr[rb[th]]; q < hp.a_ptr[rb[th + 1]]; ++q) ++ec[hp.a_col[q]];
            });
            hp.at_ptr.assign(NE + 1, 0);
            for (int e = 0; e < NE; ++e) {
                int o = hp.at_ptr[e];
                for (int th = 0; th < TT2; ++th) {
                    const int c = ecnt[(size_t)th * NE + e];
                    ecnt[(size_t)th * NE + e] = o;
                    o += c;
                }
                hp.at_ptr[e + 1] = o;
            }
            hp.at_col.resize(nnz);
            hp.at_val.resize(nnz);
            parallel_threads(TT2, [&](int th, int) {
                int* fill = &ecnt[(size_t)th * NE];
                for (int i = rb[th]; i < rb[th + 1]; ++i)
                    for (int q = hp.a_ptr[i]; q < hp.a_ptr[i + 1]; ++q) {
                        const int dst = fill[hp.a_col[q]]++;
                        hp.at_col[dst] = i;
                        hp.at_val[dst] = hp.a_val[q];
                    }
            });
        }
    }

    // ---- cached inverses: S(d) = A W diag(d)^-1 A^T (+ I for HSDE), block diagonal over components
    auto wgt = [&](int e) { return hp.prow[e] == hp.pcol[e] ? 1.0 : 2.0; };
    bool structurally_diag = true;
    for (int e = 0; e < NE && structurally_diag; ++e)
        if (hp.at_ptr[e + 1] - hp.at_ptr[e] > 1) structurally_diag = false;
    hp.minv_off.assign(hp.ncomp, 0);
    long long tot = 0;
    for (int c = 0; c < hp.ncomp; ++c) {
        const long long mc = hp.crow_ptr[c + 1] - hp.crow_ptr[c];
        if (cache_factor && !structurally_diag && mc > 8192) return CDSDP_ERR_UNSUPPORTED;
        hp.minv_off[c] = tot;
        tot += mc * mc;
    }
    hp.diag_factor = structurally_diag;
    hp.cached_factor = cache_factor;
    hp.factor_size = cache_factor ? tot : 0;
    if (cache_factor) {
        const int st = build_factor(hp, false, hp.minv);
        if (st != CDSDP_SOLVED) return st;
    }
    double nb = 0.0, nc = 0.0;
    for (int i = 0; i < m; ++i) nb += hp.b[i] * hp.b[i];
    for (int e = 0; e < NE; ++e) nc += wgt(e) * hp.c[e] * hp.c[e];
    hp.norm_b = std::sqrt(nb);
    hp.norm_c = std::sqrt(nc);
    // per component: its pattern entries and the norms of its b and c
    hp.cent_ptr.assign(hp.ncomp + 1, 0);
    for (int e = 0; e < NE; ++e) ++hp.cent_ptr[hp.comp_of_entry[e] + 1];
    for (int c = 0; c < hp.ncomp; ++c) hp.cent_ptr[c + 1] += hp.cent_ptr[c];
    hp.cent_idx.assign(NE, 0);
    {
        std::vector<int> fill(hp.cent_ptr.begin(), hp.cent_ptr.end() - 1);
        for (int e = 0; e < NE; ++e) hp.cent_idx[fill[hp.comp_of_entry[e]]++] = e;
    }
    hp.comp_nb.assign(hp.ncomp, 0.0);
    hp.comp_nc.assign(hp.ncomp, 0.0);
    for (int i = 0; i < m; ++i) hp.comp_nb[hp.comp_of_row[i]] += hp.b[i] * hp.b[i];
    for (int e = 0; e < NE; ++e) hp.comp_nc[hp.comp_of_entry[e]] += wgt(e) * hp.c[e] * hp.c[e];
    for (int c = 0; c < hp.ncomp; ++c) {
        hp.comp_nb[c] = std::sqrt(hp.comp_nb[c]);
        hp.comp_nc[c] = std::sqrt(hp.comp_nc[c]);
    }
    return CDSDP_SOLVED;
}

void scaling_factors(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col,
                     const double* A_val, const double* b, long long nnzC, const int* C_row, const int* C_col,
                     const double* C_val, int passes, std::vector<double>& d, std::vector<double>& e, double& tau,
                     double& sigma) {
    d.assign(n, 1.0);
    e.assign(m, 1.0);
    std::vector<double> rown(m), mj(n);
    auto clip = [](double x) { return std::min(1e4, std::max(1e-4, x)); };
    for (int pass = 0; pass < passes; ++pass) {
        std::fill(rown.begin(), rown.end(), 0.0);
        for (long long k = 0; k < nnzA; ++k) {
            const double a = e[A_con[k]] * d[A_row[k]] * d[A_col[k]] * A_val[k];
            rown[A_con[k]] += (A_row[k] == A_col[k] ? 1.0 : 2.0) * a * a;
        }
        for (int i = 0; i < m; ++i) {
            const double r = std::sqrt(rown[i]);
            e[i] = clip(e[i] / std::sqrt(r > 0.0 ? r : 1.0));
        }
        std::fill(mj.begin(), mj.end(), 0.0);
        for (long long k = 0; k < nnzA; ++k) {
            const double a = std::fabs(e[A_con[k]] * d[A_row[k]] * d[A_col[k]] * A_val[k]);
            mj[A_row[k]] = std::max(mj[A_row[k]], a);
            mj[A_col[k]] = std::max(mj[A_col[k]], a);
        }
        for (int j = 0; j < n; ++j) d[j] = clip(d[j] / std::sqrt(mj[j] > 0.0 ? mj[j] : 1.0));
    }
    double nb = 0.0;
    for (int i = 0; i < m; ++i) nb += (e[i] * b[i]) * (e[i] * b[i]);
    nb = std::sqrt(nb);
    tau = nb > 0.0 ? 1.0 / nb : 1.0;
    double nc = 0.0;
    for (long long k = 0; k < nnzC; ++k) {
        const double v = d[C_row[k]] * d[C_col[k]] * C_val[k];
        nc += (C_row[k] == C_col[k] ? 1.0 : 2.0) * v * v;
    }
    nc = std::sqrt(nc);
    sigma = nc > 0.0 ? 1.0 / nc : 1.0;
}

}  // namespace cdsdp_impl
