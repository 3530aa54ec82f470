// C ABI (include/cdsdp.h) of the GB300 decomposed-ADMM solver: workspace
// layout, upload, the per-iteration launch sequences of Algorithms 1-3
// (arXiv 1707.05058), the CUDA-graph while loop, and result download.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "cdsdp_internal.h"
#include "forms.cuh"
#include "cg.cuh"
#include "proj_launch.h"
#include "grad.cuh"
#include "grad_launch.h"
#include "large_launch.h"

using namespace cdsdp_dev;
using cdsdp_impl::HostProblem;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

constexpr int kNumClasses = kNumProjClasses;
static_assert(kNumClasses == CDSDP_PROJ_CLASSES, "size classes of the C ABI");
inline int class_of(int s) { return proj_class_of(s); }

struct Layout {
    // constants
    size_t c, dinv, pinv, wgt, a_ptr, a_col, a_valw, a_valu, at_ptr, at_col, at_val, b, minv, kinv, gmap, pk_off, csize,
        sc_ptr, sc_idx, zhx, zhy, atb, azhx, blist, vv_off, owner, comp_of_entry, comp_of_clique, comp_of_row, lrow,
        crow_ptr, crow_idx, ccl_ptr, ccl_idx, minv_off, cent_ptr, cent_idx, hs_nb, hs_nc, zhx_c, zhy_c, azhx_c,
        hs_zdz;
    size_t const_end;
    // state
    size_t x, t, q, s11, atuy, y, g, hh, s21, as11, ck0, ck1, ck2, vcache, part, parte, partr, scal, ctl, hist,
        comp_done, comp_iter, comp_status, comp_res, rho, cg_res, cg_p, cg_q, cg_u, cg_scal, hs_tau, hs_kappa,
        hs_gamma;
    size_t total;   // end of the state section (zeroed at every solve)
    size_t ns_off;  // dense buffers and tables of the large-clique projection (not zeroed per solve)
    size_t ws_end;  // workspace bytes
};

}  // namespace

struct cdsdp {
    HostProblem hp;
    Layout L{};
    std::vector<unsigned char> image;  // host copy of the constant section
    int cls_off[kNumClasses + 1] = {0};
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    int ws_max_iter = 0;
    Dev dev{};
    // launch shapes: grids of the pattern-entry / constraint-row kernels, lanes
    // per entry for scatters (Gs) and A^T rows (Ga), threads per A row (TPR)
    // and per row of the cached inverse (TPRM)
    int GE = 1, GR = 1, Gs = 1, Ga = 1, Gx = 1, TPR = 32, TPRM = 32;
    int TPR_auto = 32;  // TPR from the row lengths (opts.row_threads = 0)
    // Algorithm 1: compute x = t - D^-1 A^T y in its own kernel (coalesced
    // A^T rows) rather than inside the projection's gather (the default)
    bool x_split_auto = false;
    bool x_split = false;  // choice of the current solve
    // cached graph of a whole solve
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int g_form = -1;
    cdsdp_opts g_opts{};
    // last solve
    int last_form = -1, last_iters = 0, last_status = CDSDP_ERR_STATE, last_comp_mode = 0;
    std::string err;
    // profiling: event pairs around projection launches and whole iterations
    std::vector<cudaEvent_t> ev;
    bool last_profiled = false;
    double prof_proj_ms = 0.0, prof_iter_ms = 0.0;
    int prof_launches = 0;
    // per size class: an event pair around each projection launch of every
    // profiled iteration (cls_ev points at the current iteration's pairs)
    std::vector<cudaEvent_t> cls_evs;
    cudaEvent_t* cls_ev = nullptr;
    double prof_cls_ms[kNumClasses] = {0};
    int prof_cls_n[kNumClasses] = {0};
    cdsdp_impl::CmpGraph cmp_graph;  // cached step graph of the completion
    // cliques of order > 128: sign iteration on the tensor cores (large.cu)
    cdsdp_large::NsLayout ns;
    double prof_large_ms = 0.0;
    int prof_large_n = 0;
    // concurrent size classes (opts.proj_streams): side streams forked from
    // the solve's stream, classes in decreasing order of work (sum of s^3)
    cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int cls_order[kNumClasses] = {0};
};

namespace {

int fail_cuda(cdsdp* h, cudaError_t e, const char* what) {
    if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return CDSDP_ERR_CUDA;
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return fail_cuda(h, _e, #call); \
    } while (0)

// Orders of the cliques served by the sign iteration (order > 128), in clique order.
std::vector<int> large_sizes(const HostProblem& hp) {
    std::vector<int> s;
    for (size_t k = 0; k + 1 < hp.cl_off.size(); ++k) {
        const int sk = hp.cl_off[k + 1] - hp.cl_off[k];
        if (sk >= cdsdp_large::kLargeFrom) s.push_back(sk);
    }
    return s;
}

Layout make_layout(const HostProblem& hp, int max_iter) {
    Layout L{};
    size_t o = 0;
    const size_t NE = hp.prow.size(), m = hp.m, nd = hp.gmap.size(), p = hp.cl_off.size() - 1;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1)); return r; };
    const size_t nnzA = hp.a_col.size();
    const size_t minv_n = hp.minv.size();
    const size_t nc = hp.ncomp;
    L.c = take(NE * 8); L.dinv = take(NE * 8); L.pinv = take(NE * 8); L.wgt = take(NE * 8);
    L.a_ptr = take((m + 1) * 4); L.a_col = take(nnzA * 4); L.a_valw = take(nnzA * 8); L.a_valu = take(nnzA * 8);
    L.at_ptr = take((NE + 1) * 4); L.at_col = take(nnzA * 4); L.at_val = take(nnzA * 8);
    L.b = take(m * 8); L.minv = take(minv_n * 8); L.kinv = take(minv_n * 8);
    L.gmap = take(nd * 4); L.pk_off = take((p + 1) * 4); L.csize = take(p * 4);
    L.sc_ptr = take((NE + 1) * 4); L.sc_idx = take(nd * 4);
    L.zhx = take(NE * 8); L.zhy = take(m * 8); L.atb = take(NE * 8); L.azhx = take(m * 8);
    L.blist = take(p * 4);
    L.vv_off = take((p + 1) * 4);
    L.owner = take(nd);
    L.comp_of_entry = take(NE * 4); L.comp_of_clique = take(p * 4); L.comp_of_row = take(m * 4); L.lrow = take(m * 4);
    L.crow_ptr = take((nc + 1) * 4); L.crow_idx = take(m * 4); L.ccl_ptr = take((nc + 1) * 4); L.ccl_idx = take(p * 4);
    L.minv_off = take(nc * 8);
    L.cent_ptr = take((nc + 1) * 4); L.cent_idx = take(NE * 4); L.hs_nb = take(nc * 8); L.hs_nc = take(nc * 8);
    L.zhx_c = take(NE * 8); L.zhy_c = take(m * 8); L.azhx_c = take(m * 8); L.hs_zdz = take(nc * 8);
    L.const_end = o;
    L.x = take(NE * 8); L.t = take(NE * 8); L.q = take(NE * 8); L.s11 = take(NE * 8); L.atuy = take(NE * 8);
    L.y = take(m * 8); L.g = take(m * 8); L.hh = take(m * 8); L.s21 = take(m * 8); L.as11 = take(m * 8);
    L.ck0 = take(nd * 8); L.ck1 = take(nd * 8); L.ck2 = take(nd * 8);
    size_t nvv = 0;
    for (size_t k = 0; k + 1 < hp.cl_off.size(); ++k) {
        const size_t sk = hp.cl_off[k + 1] - hp.cl_off[k];
        nvv += sk * sk;
    }
    L.vcache = take(nvv * 8);
    L.part = take(p * PART_COLS * 8);
    L.parte = take((size_t)NBLK_E * PART_COLS * 8);
    L.partr = take((size_t)NBLK_R * PART_COLS * 8);
    L.scal = take(SC_WORDS * 8);
    L.ctl = take(CTL_WORDS * 4);
    L.hist = take((size_t)std::max(max_iter, 1) * HIST_COLS * 8);
    L.comp_done = take(nc * 4); L.comp_iter = take(nc * 4); L.comp_status = take(nc * 4);
    L.comp_res = take(nc * HIST_COLS * 8);
    L.rho = take(nc * 8);
    L.cg_res = take(m * 8); L.cg_p = take(m * 8); L.cg_q = take(m * 8); L.cg_u = take(NE * 8);
    L.cg_scal = take(4 * 8);
    L.hs_tau = take(nc * 8); L.hs_kappa = take(nc * 8); L.hs_gamma = take(nc * 8);
    L.total = o;
    L.ns_off = o;
    L.ws_end = o + cdsdp_large::ns_layout(large_sizes(hp)).bytes;
    return L;
}

template <typename V, typename A>
void put(std::vector<unsigned char>& img, size_t off, const std::vector<V, A>& v) {
    if (!v.empty()) std::memcpy(img.data() + off, v.data(), v.size() * sizeof(V));
}

void build_image(cdsdp* h) {
    const HostProblem& hp = h->hp;
    const Layout& L = h->L;
    const int NE = (int)hp.prow.size(), p = (int)hp.cl_off.size() - 1;
    h->image.assign(L.const_end, 0);
    auto& img = h->image;
    put(img, L.c, hp.c);
    std::vector<double> dinv(NE), pinv(NE), wgt(NE), aw(hp.a_val.size());
    for (int e = 0; e < NE; ++e) {
        dinv[e] = 1.0 / hp.D[e];
        pinv[e] = 1.0 / (1.0 + 0.5 * hp.D[e]);
        wgt[e] = hp.prow[e] == hp.pcol[e] ? 1.0 : 2.0;
    }
    for (size_t q = 0; q < hp.a_val.size(); ++q) aw[q] = wgt[hp.a_col[q]] * hp.a_val[q];
    put(img, L.dinv, dinv); put(img, L.pinv, pinv); put(img, L.wgt, wgt);
    put(img, L.a_ptr, hp.a_ptr); put(img, L.a_col, hp.a_col); put(img, L.a_valw, aw); put(img, L.a_valu, hp.a_val);
    put(img, L.at_ptr, hp.at_ptr); put(img, L.at_col, hp.at_col); put(img, L.at_val, hp.at_val);
    put(img, L.b, hp.b); put(img, L.minv, hp.minv); put(img, L.kinv, hp.kinv);
    put(img, L.gmap, hp.gmap); put(img, L.pk_off, hp.pk_off);
    std::vector<int> cs(p);
    for (int k = 0; k < p; ++k) cs[k] = hp.cl_off[k + 1] - hp.cl_off[k];
    put(img, L.csize, cs);
    put(img, L.sc_ptr, hp.sc_ptr); put(img, L.sc_idx, hp.sc_idx);
    put(img, L.zhx, hp.zhat_x); put(img, L.zhy, hp.zhat_y); put(img, L.atb, hp.atb); put(img, L.azhx, hp.a_zhat_x);
    // clique lists by size class
    std::vector<int> blist;
    for (int c = 0; c < kNumClasses; ++c) {
        h->cls_off[c] = (int)blist.size();
        for (int k = 0; k < p; ++k)
            if (class_of(cs[k]) == c) blist.push_back(k);
    }
    h->cls_off[kNumClasses] = (int)blist.size();
    put(img, L.blist, blist);
    std::vector<int> vv(p + 1, 0);
    for (int k = 0; k < p; ++k) vv[k + 1] = vv[k] + cs[k] * cs[k];
    put(img, L.vv_off, vv);
    std::vector<unsigned char> own(hp.gmap.size(), 0);
    for (int e = 0; e < NE; ++e)
        if (hp.sc_ptr[e + 1] > hp.sc_ptr[e]) own[hp.sc_idx[hp.sc_ptr[e]]] = 1;
    put(img, L.owner, own);
    put(img, L.comp_of_entry, hp.comp_of_entry); put(img, L.comp_of_clique, hp.comp_of_clique);
    put(img, L.comp_of_row, hp.comp_of_row); put(img, L.lrow, hp.lrow);
    put(img, L.crow_ptr, hp.crow_ptr); put(img, L.crow_idx, hp.crow_idx);
    put(img, L.ccl_ptr, hp.ccl_ptr); put(img, L.ccl_idx, hp.ccl_idx); put(img, L.minv_off, hp.minv_off);
    put(img, L.cent_ptr, hp.cent_ptr); put(img, L.cent_idx, hp.cent_idx);
    put(img, L.hs_nb, hp.comp_nb); put(img, L.hs_nc, hp.comp_nc);
}

void make_dev(cdsdp* h) {
    const HostProblem& hp = h->hp;
    const Layout& L = h->L;
    unsigned char* w = h->ws;
    Dev& d = h->dev;
    d.n = hp.n; d.m = hp.m; d.NE = (int)hp.prow.size(); d.p = (int)hp.cl_off.size() - 1; d.nd = (int)hp.gmap.size();
    d.diag_factor = hp.diag_factor ? 1 : 0;
    d.c = (const double*)(w + L.c); d.dinv = (const double*)(w + L.dinv); d.pinv = (const double*)(w + L.pinv);
    d.wgt = (const double*)(w + L.wgt);
    d.a_ptr = (const int*)(w + L.a_ptr); d.a_col = (const int*)(w + L.a_col); d.a_valw = (const double*)(w + L.a_valw);
    d.a_valu = (const double*)(w + L.a_valu);
    d.wstore = nullptr; d.wstore_count = 0;
    d.at_ptr = (const int*)(w + L.at_ptr); d.at_col = (const int*)(w + L.at_col); d.at_val = (const double*)(w + L.at_val);
    d.b = (const double*)(w + L.b); d.minv = (const double*)(w + L.minv); d.kinv = (const double*)(w + L.kinv);
    d.gmap = (const int*)(w + L.gmap); d.pk_off = (const int*)(w + L.pk_off); d.csize = (const int*)(w + L.csize);
    d.sc_ptr = (const int*)(w + L.sc_ptr); d.sc_idx = (const int*)(w + L.sc_idx);
    d.zhx = (const double*)(w + L.zhx); d.zhy = (const double*)(w + L.zhy);
    d.atb = (const double*)(w + L.atb); d.azhx = (const double*)(w + L.azhx);
    d.zeta_dot_zhat = hp.zeta_dot_zhat; d.norm_b = hp.norm_b; d.norm_c = hp.norm_c;
    d.x = (double*)(w + L.x); d.t = (double*)(w + L.t); d.q = (double*)(w + L.q); d.s11 = (double*)(w + L.s11);
    d.atuy = (double*)(w + L.atuy);
    d.y = (double*)(w + L.y); d.g = (double*)(w + L.g); d.hh = (double*)(w + L.hh); d.s21 = (double*)(w + L.s21);
    d.as11 = (double*)(w + L.as11);
    d.ck0 = w + L.ck0; d.ck1 = w + L.ck1; d.ck2 = w + L.ck2;
    d.vcache = w + L.vcache; d.vv_off = (const int*)(w + L.vv_off);
    d.owner = (const unsigned char*)(w + L.owner);
    d.part = (double*)(w + L.part); d.parte = (double*)(w + L.parte); d.partr = (double*)(w + L.partr);
    d.scal = (double*)(w + L.scal); d.ctl = (int*)(w + L.ctl); d.hist = (double*)(w + L.hist);
    d.max_iter = h->ws_max_iter;
    d.ncomp = hp.ncomp;
    d.rows_contig = hp.rows_contiguous ? 1 : 0;
    d.comp_mode = 0;
    d.comp_of_entry = (const int*)(w + L.comp_of_entry); d.comp_of_clique = (const int*)(w + L.comp_of_clique);
    d.comp_of_row = (const int*)(w + L.comp_of_row); d.lrow = (const int*)(w + L.lrow);
    d.crow_ptr = (const int*)(w + L.crow_ptr); d.crow_idx = (const int*)(w + L.crow_idx);
    d.ccl_ptr = (const int*)(w + L.ccl_ptr); d.ccl_idx = (const int*)(w + L.ccl_idx);
    d.minv_off = (const long long*)(w + L.minv_off);
    d.comp_done = (int*)(w + L.comp_done); d.comp_iter = (int*)(w + L.comp_iter);
    d.comp_status = (int*)(w + L.comp_status); d.comp_res = (double*)(w + L.comp_res);
    d.rho = (double*)(w + L.rho);
    d.cg_res = (double*)(w + L.cg_res); d.cg_p = (double*)(w + L.cg_p); d.cg_q = (double*)(w + L.cg_q);
    d.cg_u = (double*)(w + L.cg_u); d.cg_scal = (double*)(w + L.cg_scal);
    d.cg_tol = 0.0; d.cg_max = 0;
    d.hs_tau = (double*)(w + L.hs_tau); d.hs_kappa = (double*)(w + L.hs_kappa); d.hs_gamma = (double*)(w + L.hs_gamma);
    d.hs_zdz = (const double*)(w + L.hs_zdz); d.hs_nb = (const double*)(w + L.hs_nb);
    d.hs_nc = (const double*)(w + L.hs_nc);
    d.cent_ptr = (const int*)(w + L.cent_ptr); d.cent_idx = (const int*)(w + L.cent_idx);
    auto pow2_clamp = [](double x, int lo, int hi) {
        int v = lo;
        while (v < hi && v < x) v <<= 1;
        return v;
    };
    const double avg_sc = d.NE ? double(d.nd) / d.NE : 1.0;
    const double avg_at = d.NE ? double(hp.a_col.size()) / d.NE : 1.0;
    const double avg_a = d.m ? double(hp.a_col.size()) / d.m : 1.0;
    h->Gs = pow2_clamp(avg_sc / 2.0, 1, 32);
    h->Ga = pow2_clamp(std::max(avg_at, avg_sc) / 3.0, 1, 32);
    h->Gx = pow2_clamp(avg_at / 6.0, 1, 32);  // lanes per A^T row in the separate x-update
    h->TPR = h->TPR_auto = pow2_clamp(avg_a / 4.0, 32, RTHREADS);
    // The separate kernel forms each x_e once (in float64, whose throughput is
    // low on this GPU); inside the gather it is formed once per clique holding e.
    h->x_split_auto = true;
    h->x_split = h->x_split_auto;
    int max_mc = 0;
    for (int c = 0; c < hp.ncomp; ++c) max_mc = std::max(max_mc, hp.crow_ptr[c + 1] - hp.crow_ptr[c]);
    // threads per row of the cached inverse: about 16 entries a thread (rows of
    // a few hundred entries take one warp, reduced without a barrier)
    h->TPRM = hp.diag_factor ? 32 : pow2_clamp(max_mc / 16.0, 32, RTHREADS);
    const int G = std::max(h->Gs, h->Ga);
    h->GE = std::max(1, std::min(NBLK_E, (int)(((long long)d.NE * G + ETHREADS - 1) / ETHREADS)));
    const int TP = std::max(h->TPR, h->TPRM);
    h->GR = std::max(1, std::min(NBLK_R, (d.m + RTHREADS / TP - 1) / (RTHREADS / TP)));
}

// ---- scatter dispatch -------------------------------------------------------

// H^T (...) onto the pattern: in packed-position order when the entries
// average fewer than two cliques each (one lane per entry), else one group of
// lanes per entry.
template <typename T>
void launch_scatter(const cdsdp* h, const Dev& d, const T* P, const T* Q, double alpha, double beta, double gamma,
                    int alpha_rho, int gamma_rho, const double* scale, double* out, int check_stop, cudaStream_t st) {
    if (h->Gs == 1) {
        const int grid = (int)std::max<long long>(1, std::min<long long>(152LL * 16, ((long long)d.nd + ETHREADS - 1) / ETHREADS));
        k_scatter_owner<T><<<grid, ETHREADS, 0, st>>>(d, P, Q, alpha, beta, gamma, alpha_rho, gamma_rho, scale, out,
                                                      check_stop);
    } else {
        k_scatter<T><<<h->GE, ETHREADS, 0, st>>>(d, P, Q, alpha, beta, gamma, alpha_rho, gamma_rho, scale, out,
                                                check_stop, h->Gs);
    }
}

// ---- projection dispatch ----------------------------------------------------

template <typename T>
cudaError_t launch_projection(cdsdp* h, int form, const cdsdp_opts& o, const FinishArgs& fa, cudaStream_t st) {
    const int* bl = (const int*)(h->ws + h->L.blist);
    ProjArgs pa;
    pa.tolrel = sizeof(T) == 4 ? 1.2e-7 : 2.3e-16;
    pa.max_sweeps = o.jacobi_max_sweeps;
    pa.warm_start = o.warm_start > 0 ? 1 : 0;
    pa.restart = o.warm_start > 0 ? o.warm_start : 1;
    int last = -1;
    for (int c = 0; c < kNumClasses; ++c)
        if (h->cls_off[c + 1] > h->cls_off[c]) last = c;
    const bool large = h->ns.nb > 0;
    if (large) last = -1;  // the large cliques' reduction finishes the iteration
    cudaError_t e = cudaSuccess;
    pa.row_off = 0;
    pa.warps_div = o.proj_warps_div;
    pa.x_ready = (form == 0 && h->x_split) ? 1 : 0;
    pa.cta_variant = o.proj_cta_kernel;
    // first partial-table row of each class (class order), then the launches
    int row0[kNumClasses + 1];
    for (int c = 0; c < kNumClasses; ++c) {
        const int nl = h->cls_off[c + 1] - h->cls_off[c];
        row0[c] = pa.row_off;
        if (nl > 0) pa.row_off += proj_launch_grid(c, nl, sizeof(T) == 4, pa.warps_div);
    }
    row0[kNumClasses] = pa.row_off;
    // Concurrent classes need stopping tests that run after all of them (the
    // component mode's own kernel): fork side streams, join them at the end.
    int ns = 1;
    if (h->dev.comp_mode && o.proj_streams > 1 && h->side[0]) {
        int work = large ? 1 : 0;
        for (int c = 0; c < kNumClasses; ++c) work += h->cls_off[c + 1] > h->cls_off[c] ? 1 : 0;
        ns = std::min(std::min(o.proj_streams, 4), work);
    }
    if (ns > 1) {
        if ((e = cudaEventRecord(h->fork_ev, st)) != cudaSuccess) return e;
        for (int i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(h->side[i], h->fork_ev, 0)) != cudaSuccess) return e;
    }
    int q = 0;
    for (int i = 0; i < kNumClasses && e == cudaSuccess; ++i) {
        const int c = ns > 1 ? h->cls_order[i] : i;
        const int* list = bl + h->cls_off[c];
        const int nl = h->cls_off[c + 1] - h->cls_off[c];
        if (nl <= 0) continue;
        cudaStream_t sc = ns > 1 ? h->side[q++ % ns] : st;
        FinishArgs f = fa;
        f.enabled = (c == last) ? fa.enabled : 0;  // the last launch finishes the iteration
        ProjArgs pc = pa;
        pc.row_off = row0[c];
        if (h->cls_ev) cudaEventRecord(h->cls_ev[2 * c], sc);
        e = sizeof(T) == 4 ? launch_proj_f32(form, c, h->dev, list, nl, pc, f, sc)
                           : launch_proj_f64(form, c, h->dev, list, nl, pc, f, sc);
        if (h->cls_ev) cudaEventRecord(h->cls_ev[2 * c + 1], sc);
    }
    if (large && e == cudaSuccess) {  // float clique state only (FP64 refuses these orders)
        cudaStream_t sc = ns > 1 ? h->side[q++ % ns] : st;
        if (h->cls_ev) cudaEventRecord(h->cls_ev[2 * kNumClasses], sc);
        e = cdsdp_large::large_step(form, h->dev, h->ns, h->ws + h->L.ns_off, row0[kNumClasses], fa, sc);
        if (h->cls_ev) cudaEventRecord(h->cls_ev[2 * kNumClasses + 1], sc);
    }
    if (ns > 1) {
        for (int i = 0; i < ns; ++i) {
            const cudaError_t e2 = cudaEventRecord(h->join_ev[i], h->side[i]);
            const cudaError_t e3 = cudaStreamWaitEvent(st, h->join_ev[i], 0);
            if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
        }
    }
    return e;
}

// ---- one ADMM iteration -----------------------------------------------------

// y from (A W D^-1 A^T) y = d.g by conjugate gradient (Section 4.1.1), warm
// start from the y in place; leaves the <b, y> partial of k_gemv.
void launch_cg(cdsdp* h, const cdsdp_opts& o, cudaStream_t st) {
    Dev& d = h->dev;
    k_cg_atp<<<h->GE, ETHREADS, 0, st>>>(d, d.y, h->Gx, 0);
    k_cg_aw<<<h->GR, RTHREADS, 0, st>>>(d, h->TPR, 0);
    k_cg_init<<<1, CG_THREADS, 0, st>>>(d, d.g);
    for (int s = 0; s < o.cg_max_steps; ++s) {
        k_cg_atp<<<h->GE, ETHREADS, 0, st>>>(d, d.cg_p, h->Gx, 1);
        k_cg_aw<<<h->GR, RTHREADS, 0, st>>>(d, h->TPR, 1);
        k_cg_update<<<1, CG_THREADS, 0, st>>>(d);
    }
    k_cg_finish<<<1, CG_THREADS, 0, st>>>(d, 0, h->GR);
}

template <typename T>
cudaError_t launch_iteration(cdsdp* h, int form, const cdsdp_opts& o, cudaStream_t st, int use_cond,
                             cudaGraphConditionalHandle hnd, cudaEvent_t ev0, cudaEvent_t ev1) {
    Dev& d = h->dev;
    const int GE = h->GE, GR = h->GR, PG = std::max(1, std::min((d.p + 3) / 4, 152 * 32));
    FinishArgs fa;
    fa.eps = o.eps;
    fa.mu = o.rho_mu;
    fa.nu = o.rho_nu;
    fa.adapt_every = o.adaptive_rho;
    fa.nbe = GE;
    fa.nbr = GR;
    // rows of the clique partial table written this iteration: one per block of
    // every projection launch (and, for Algorithm 2, of the v/lambda kernel)
    int prow = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        const int nl = h->cls_off[c + 1] - h->cls_off[c];
        if (nl > 0) prow += proj_launch_grid(c, nl, sizeof(T) == 4, o.proj_warps_div);
    }
    prow += h->ns.nb;  // one row per large clique
    fa.npart = std::min(d.p, form == 1 ? std::max(prow, PG) : prow);
    fa.enabled = 1;
    fa.use_cond = use_cond;
    fa.hnd = hnd;
    // with independent components stopping on their own, a separate kernel
    // (one block per component) runs the tests after the last update
    FinishArgs fin = fa;
    if (d.comp_mode) fin.enabled = 0;
    cudaError_t e;
    if (form == 0) {  // Algorithm 1; the projection computes x on the fly and its last block the stopping test
        launch_scatter<T>(h, d, (const T*)d.ck0, (const T*)d.ck1, -1.0, 1.0, 1.0, 1, 1, d.dinv, d.t, 1, st);
        k_rows_aw<<<GR, RTHREADS, 0, st>>>(d, d.t, -1.0, 0, d.g, h->TPR);
        if (o.linear_solver == 1) launch_cg(h, o, st);
        else k_gemv<<<GR, RTHREADS, 0, st>>>(d, d.minv, d.g, d.y, 0, h->TPRM);
        if (h->x_split) k_xupd<<<GE, ETHREADS, 0, st>>>(d, d.t, d.y, d.x, h->Gx, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ev0) cudaEventRecord(ev0, st);
        if ((e = launch_projection<T>(h, 0, o, fin, st)) != cudaSuccess) return e;
        if (ev1) cudaEventRecord(ev1, st);
        if (d.comp_mode) k_finish_components<<<d.ncomp, 256, 0, st>>>(d, 0, fa);
    } else if (form == 1) {  // Algorithm 2; the v/lambda kernel's last block runs the stopping test
        if (ev0) cudaEventRecord(ev0, st);
        FinishArgs none = fa;
        none.enabled = 0;
        if ((e = launch_projection<T>(h, 1, o, none, st)) != cudaSuccess) return e;
        if (ev1) cudaEventRecord(ev1, st);
        launch_scatter<T>(h, d, (const T*)d.ck0, (const T*)d.ck2, 1.0, -1.0, 1.0, 0, 1, d.dinv, d.t, 1, st);
        k_rows_aw<<<GR, RTHREADS, 0, st>>>(d, d.t, 1.0, 1, d.g, h->TPR);
        if (o.linear_solver == 1) launch_cg(h, o, st);
        else k_gemv<<<GR, RTHREADS, 0, st>>>(d, d.minv, d.g, d.y, 0, h->TPRM);
        k_xupd<<<GE, ETHREADS, 0, st>>>(d, d.t, d.y, d.x, h->Ga, 1);
        k_vlam_dual<T><<<PG, 128, 0, st>>>(d, fin);
        if (d.comp_mode) k_finish_components<<<d.ncomp, 256, 0, st>>>(d, 1, fa);
    } else {  // Algorithm 3; gamma/tau/kappa in sigma21's last block, stopping test in row_update's
        k_hsde_eta<T><<<GE, ETHREADS, 0, st>>>(d, h->Gs);
        k_rows_aw<<<GR, RTHREADS, 0, st>>>(d, d.q, 0.0, 0, d.g, h->TPR);
        k_gemv<<<GR, RTHREADS, 0, st>>>(d, d.kinv, d.g, d.hh, -1, h->TPRM);
        k_hsde_sigma11<<<GE, ETHREADS, 0, st>>>(d, h->Ga);
        k_hsde_sigma21<<<GR, RTHREADS, 0, st>>>(d, h->TPR, GE);
        if (d.comp_mode) k_hsde_gamma_components<<<d.ncomp, 256, 0, st>>>(d);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ev0) cudaEventRecord(ev0, st);
        FinishArgs none = fa;
        none.enabled = 0;
        if ((e = launch_projection<T>(h, 2, o, none, st)) != cudaSuccess) return e;
        if (ev1) cudaEventRecord(ev1, st);
        k_hsde_entry_update<T><<<GE, ETHREADS, 0, st>>>(d, h->Ga);
        k_hsde_row_update<<<GR, RTHREADS, 0, st>>>(d, fa);
        if (d.comp_mode) k_finish_hsde_components<<<d.ncomp, 256, 0, st>>>(d, fa);
    }
    return cudaGetLastError();
}

cudaError_t launch_iteration_any(cdsdp* h, int form, const cdsdp_opts& o, cudaStream_t st, int use_cond,
                                 cudaGraphConditionalHandle hnd, cudaEvent_t ev0 = nullptr,
                                 cudaEvent_t ev1 = nullptr) {
    return o.precision == CDSDP_FP64 ? launch_iteration<double>(h, form, o, st, use_cond, hnd, ev0, ev1)
                                     : launch_iteration<float>(h, form, o, st, use_cond, hnd, ev0, ev1);
}

bool same_opts(const cdsdp_opts& a, const cdsdp_opts& b) {
    return a.eps == b.eps && a.max_iter == b.max_iter && a.rho == b.rho && a.precision == b.precision &&
           a.jacobi_max_sweeps == b.jacobi_max_sweeps && a.warm_start == b.warm_start &&
           a.component_stop == b.component_stop && a.adaptive_rho == b.adaptive_rho && a.rho_mu == b.rho_mu &&
           a.rho_nu == b.rho_nu && a.x_update == b.x_update && a.proj_warps_div == b.proj_warps_div &&
           a.linear_solver == b.linear_solver && a.cg_tol == b.cg_tol && a.cg_max_steps == b.cg_max_steps &&
           a.proj_streams == b.proj_streams && a.proj_cta_kernel == b.proj_cta_kernel &&
           a.row_threads == b.row_threads;
}

void drop_graph(cdsdp* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->g_form = -1;
}

// The whole solve as one graph: a while node whose body is one iteration;
// the iteration's last kernel clears the condition when the solve is done.
int build_graph(cdsdp* h, int form, const cdsdp_opts& o) {
    drop_graph(h);
    CK(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle hnd;
    CK(cudaGraphConditionalHandleCreate(&hnd, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = launch_iteration_any(h, form, o, cs, 1, hnd);
        e = cudaStreamEndCapture(cs, &body);
        if (e2 != cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { drop_graph(h); return fail_cuda(h, e, "graph capture"); }
    e = cudaGraphInstantiate(&h->gexec, h->graph, 0);
    if (e != cudaSuccess) { drop_graph(h); return fail_cuda(h, e, "cudaGraphInstantiate"); }
    h->g_form = form;
    h->g_opts = o;
    return CDSDP_SOLVED;
}

int check_opts(const cdsdp* h, const cdsdp_opts& o) {
    if (!(o.eps >= 0) || o.max_iter < 1 || !(o.rho > 0) || o.jacobi_max_sweeps < 1 || o.check_every < 1) return CDSDP_ERR_ARG;
    if (o.precision != CDSDP_FP32_PROJECTION && o.precision != CDSDP_FP64) return CDSDP_ERR_ARG;
    if (o.max_iter > h->ws_max_iter) return CDSDP_ERR_ARG;
    if (o.warm_start < 0) return CDSDP_ERR_ARG;
    if (o.component_stop != 0 && o.component_stop != 1) return CDSDP_ERR_ARG;
    if (o.adaptive_rho < 0 || !(o.rho_mu >= 1.0) || !(o.rho_nu >= 1.0)) return CDSDP_ERR_ARG;
    if (o.x_update < 0 || o.x_update > 2) return CDSDP_ERR_ARG;
    if (o.proj_warps_div != 1 && o.proj_warps_div != 2 && o.proj_warps_div != 4) return CDSDP_ERR_ARG;
    if (o.linear_solver != 0 && o.linear_solver != 1) return CDSDP_ERR_ARG;
    if (!(o.cg_tol >= 0.0) || !std::isfinite(o.cg_tol) || o.cg_max_steps < 0 || o.cg_max_steps > 1024)
        return CDSDP_ERR_ARG;
    if (o.proj_streams < 1 || o.proj_streams > 4) return CDSDP_ERR_ARG;
    if (o.proj_cta_kernel != 0 && o.proj_cta_kernel != 1) return CDSDP_ERR_ARG;
    if (o.row_threads != 0 && o.row_threads != 32 && o.row_threads != 64 && o.row_threads != 128 &&
        o.row_threads != 256)
        return CDSDP_ERR_ARG;
    if (o.precision == CDSDP_FP64 && h->hp.max_clique > kMaxOrderF64) return CDSDP_ERR_UNSUPPORTED;
    return CDSDP_SOLVED;
}

// Algorithm 3's cached inverse and constants are built on the first HSDE solve
// (host) and copied into their slots of the bound workspace.
int ensure_hsde(cdsdp* h, cudaStream_t st) {
    if (h->hp.hsde_ready) return CDSDP_SOLVED;
    int rc;
    try {
        rc = cdsdp_impl::build_hsde_constants(h->hp);
    } catch (const std::exception&) {  // allocation or thread creation failed
        rc = CDSDP_ERR_NOMEM;
    }
    if (rc != CDSDP_SOLVED) return rc;
    const HostProblem& hp = h->hp;
    const Layout& L = h->L;
    put(h->image, L.kinv, hp.kinv);
    put(h->image, L.zhx, hp.zhat_x);
    put(h->image, L.zhy, hp.zhat_y);
    put(h->image, L.atb, hp.atb);
    put(h->image, L.azhx, hp.a_zhat_x);
    put(h->image, L.zhx_c, hp.zhat_x_c);
    put(h->image, L.zhy_c, hp.zhat_y_c);
    put(h->image, L.azhx_c, hp.a_zhat_x_c);
    put(h->image, L.hs_zdz, hp.zdz_c);
    const size_t sections[9][2] = {{L.kinv, hp.kinv.size() * 8}, {L.zhx, hp.zhat_x.size() * 8},
                                   {L.zhy, hp.zhat_y.size() * 8}, {L.atb, hp.atb.size() * 8},
                                   {L.azhx, hp.a_zhat_x.size() * 8}, {L.zhx_c, hp.zhat_x_c.size() * 8},
                                   {L.zhy_c, hp.zhat_y_c.size() * 8}, {L.azhx_c, hp.a_zhat_x_c.size() * 8},
                                   {L.hs_zdz, hp.zdz_c.size() * 8}};
    for (const auto& sec : sections)
        if (sec[1]) CK(cudaMemcpyAsync(h->ws + sec[0], h->image.data() + sec[0], sec[1], cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    h->dev.zeta_dot_zhat = hp.zeta_dot_zhat;
    return CDSDP_SOLVED;
}

// Map a solution of the scaled problem (Section 7.1.3) back on the host:
// X = D Xbar D / tau, y_i = e_i ybar_i / sigma, Z = D^-1 Zbar D^-1 / sigma,
// entrywise on the lower pattern.
void unscale_results(const HostProblem& hp, double* X, double* y, double* Z) {
    const size_t NE = hp.prow.size();
    for (size_t k = 0; k < NE; ++k) {
        const double dd = hp.sc_d[hp.prow[k]] * hp.sc_d[hp.pcol[k]];
        if (X) X[k] *= dd / hp.sc_tau_v[hp.prow[k]];
        if (Z) Z[k] /= dd * hp.sc_sigma_v[hp.prow[k]];
    }
    if (y)
        for (int i = 0; i < hp.m; ++i) y[i] *= hp.sc_e[i] / hp.sc_sigma_r[i];
}

// Certificates of the scaled problem mapped back.  A primal infeasibility
// certificate ybar with bbar^T ybar = 1 gives y_i = tau e_i ybar_i with
// b^T y = 1; a dual one Xbar with Cbar . Xbar = -1 gives X = sigma D Xbar D
// with C . X = -1, the normalisations of an unscaled solve.
void unscale_cert(const HostProblem& hp, int status, double* cert) {
    if (status == CDSDP_PRIMAL_INFEASIBLE) {
        for (int i = 0; i < hp.m; ++i) cert[i] *= hp.sc_tau_r[i] * hp.sc_e[i];
    } else if (status == CDSDP_DUAL_INFEASIBLE) {
        const size_t NE = hp.prow.size();
        for (size_t k = 0; k < NE; ++k)
            cert[k] *= hp.sc_sigma_v[hp.prow[k]] * hp.sc_d[hp.prow[k]] * hp.sc_d[hp.pcol[k]];
    }
}

int copy_results(cdsdp* h, cudaStream_t st, double* X, double* y, double* Z, double* hist, double* cert) {
    Dev& d = h->dev;
    const int form = h->last_form;
    const int NE = d.NE, m = d.m;
    const bool fp64 = h->g_opts.precision == CDSDP_FP64;
    double* tmpE = d.t;  // scratch after the solve
    double* tmpM = d.g;
    const double* tau = d.scal + SC_TAU;
    const bool hs_comp = form == 2 && h->last_comp_mode;  // tau per component
    if (X) {
        if (form == 0) k_scale_out<<<64, 256, 0, st>>>(NE, d.x, 1.0, nullptr, tmpE);
        else if (form == 1) k_scale_rho<<<64, 256, 0, st>>>(d, NE, d.x, -1.0, 0, tmpE);
        else if (hs_comp) k_scale_hs_tau<<<64, 256, 0, st>>>(d, NE, d.x, 0, tmpE);
        else k_scale_out<<<64, 256, 0, st>>>(NE, d.x, 1.0, tau, tmpE);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(X, tmpE, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (y) {
        if (form == 0) k_scale_rho<<<8, 256, 0, st>>>(d, m, d.y, -1.0, 1, tmpM);
        else if (form == 1) k_scale_out<<<8, 256, 0, st>>>(m, d.y, 1.0, nullptr, tmpM);
        else if (hs_comp) k_scale_hs_tau<<<8, 256, 0, st>>>(d, m, d.y, 1, tmpM);
        else k_scale_out<<<8, 256, 0, st>>>(m, d.y, 1.0, tau, tmpM);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(y, tmpM, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (Z) {
        const void* src = form == 0 ? d.ck1 : (form == 1 ? d.ck0 : d.ck1);  // lambda, z, v_z
        if (fp64) launch_scatter<double>(h, d, (const double*)src, nullptr, 0.0, 1.0, 0.0, 0, 0, nullptr, tmpE, 0, st);
        else launch_scatter<float>(h, d, (const float*)src, nullptr, 0.0, 1.0, 0.0, 0, 0, nullptr, tmpE, 0, st);
        if (form == 2 && hs_comp) k_scale_hs_tau<<<64, 256, 0, st>>>(d, NE, tmpE, 0, tmpE);
        else if (form == 2) k_scale_out<<<64, 256, 0, st>>>(NE, tmpE, 1.0, tau, tmpE);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(Z, tmpE, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (h->hp.scaled) unscale_results(h->hp, X, y, Z);
    if (hist && h->last_iters > 0) {
        CK(cudaMemcpyAsync(hist, d.hist, (size_t)h->last_iters * HIST_COLS * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (cert && form == 2 && !hs_comp) {
        if (h->last_status == CDSDP_PRIMAL_INFEASIBLE) {  // u_y / (b^T u_y)
            double* dots = d.scal + 8;
            k_dot<<<1, 256, 0, st>>>(m, d.y, d.b, nullptr, dots);
            k_scale_out<<<8, 256, 0, st>>>(m, d.y, 1.0, dots, tmpM, 2);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(cert, tmpM, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        } else if (h->last_status == CDSDP_DUAL_INFEASIBLE) {  // -u_x / (c^T u_x)
            double* dots = d.scal + 8;
            k_dot<<<1, 256, 0, st>>>(NE, d.x, d.c, d.wgt, dots);
            k_scale_out<<<64, 256, 0, st>>>(NE, d.x, -1.0, dots, tmpE, 2);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(cert, tmpE, NE * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        if (h->hp.scaled) unscale_cert(h->hp, h->last_status, cert);
    }
    return CDSDP_SOLVED;
}

}  // namespace

// ---- differentiation through unrolled Algorithm 1 -------------------------

struct GradLayout {
    size_t ckpt, wstore, xkbar, lambar, hxbar, lamprev, xbar, u, sbar, ybar, rbar, total;
    int nseg;
};

GradLayout make_grad_layout(const Dev& d, int iters, int ckpt_every, bool fp32) {
    GradLayout G{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + std::max<size_t>(bytes, 1)); return r; };
    const size_t ts = fp32 ? 4 : 8, nd = d.nd, NE = d.NE, m = d.m;
    G.nseg = (iters + ckpt_every - 1) / ckpt_every;
    G.ckpt = take((size_t)G.nseg * 2 * nd * ts);
    G.wstore = take((size_t)ckpt_every * nd * ts);
    G.xkbar = take(nd * 8); G.lambar = take(nd * 8); G.hxbar = take(nd * 8); G.lamprev = take(nd * 8);
    G.xbar = take(NE * 8); G.u = take(NE * 8); G.sbar = take(NE * 8);
    G.ybar = take(m * 8); G.rbar = take(m * 8);
    G.total = o;
    return G;
}

int check_unrolled(cdsdp* h, const cdsdp_opts& o, int iters, int ckpt_every) {
    if (!h->ws) return CDSDP_ERR_STATE;
    if (iters < 1 || ckpt_every < 1 || !(o.rho > 0) || o.jacobi_max_sweeps < 1) return CDSDP_ERR_ARG;
    if (o.precision != CDSDP_FP32_PROJECTION && o.precision != CDSDP_FP64) return CDSDP_ERR_ARG;
    if (h->hp.max_clique > kMaxWarpOrder) return CDSDP_ERR_UNSUPPORTED;
    if (h->hp.scaled) return CDSDP_ERR_UNSUPPORTED;  // c and b would be in scaled units
    if (!h->hp.cached_factor) return CDSDP_ERR_UNSUPPORTED;  // the reverse pass applies the inverse
    if (ckpt_every > h->ws_max_iter) return CDSDP_ERR_ARG;
    return CDSDP_SOLVED;
}

// Run `len` iterations of Algorithm 1 (no early stop) with the device view dd.
int run_segment(cdsdp* h, Dev dd, const cdsdp_opts& o, int len, cudaStream_t st) {
    const Dev saved = h->dev;
    h->dev = dd;
    k_reset_ctl<<<1, 32, 0, st>>>(dd, o.rho);
    cudaError_t e = cudaGetLastError();
    for (int it = 0; it < len && e == cudaSuccess; ++it)
        e = launch_iteration_any(h, 0, o, st, 0, cudaGraphConditionalHandle{});
    h->dev = saved;
    return e == cudaSuccess ? CDSDP_SOLVED : fail_cuda(h, e, "unrolled iteration");
}

cdsdp_opts unrolled_opts(const cdsdp_opts* opts) {
    cdsdp_opts o;
    if (opts) o = *opts; else cdsdp_default_opts(&o);
    o.eps = 0.0;        // fixed number of iterations
    o.warm_start = 0;   // replays must repeat the forward bit for bit
    o.use_graph = 0;
    o.profile = 0;
    o.adaptive_rho = 0;  // the reverse pass assumes one fixed rho
    o.linear_solver = 0;  // and the cached inverse
    return o;
}

// =============================================================================
// C ABI

extern "C" {

void cdsdp_default_opts(cdsdp_opts* o) {
    if (!o) return;
    o->eps = 1e-4;
    o->max_iter = 2000;
    o->rho = 1.0;
    o->precision = CDSDP_FP32_PROJECTION;
    o->use_graph = 1;
    o->check_every = 50;
    o->jacobi_max_sweeps = 30;
    o->warm_start = 16;
    o->profile = 0;
    o->component_stop = 1;
    o->adaptive_rho = 0;
    o->rho_mu = 2.0;
    o->rho_nu = 10.0;
    o->x_update = 0;
    o->proj_warps_div = 1;
    o->linear_solver = 0;
    o->cg_tol = 1e-10;
    o->cg_max_steps = 5;
    o->proj_streams = 4;
    o->proj_cta_kernel = 1;
    o->row_threads = 0;
}

namespace {

// Both setup entry points: scale_passes < 0 sets the data up as given;
// flags as cdsdp_setup_flags.
int setup_common(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col,
                 const double* A_val, const double* b, long long nnzC, const int* C_row, const int* C_col,
                 const double* C_val, long long nnzP, const int* P_row, const int* P_col, int scale_passes,
                 unsigned flags, cdsdp** out, int count = 0, const int* sdp_n = nullptr,
                 const int* sdp_m = nullptr) {
    if (!out) return CDSDP_ERR_ARG;
    *out = nullptr;
    if (flags & ~(unsigned)(CDSDP_SETUP_NO_FACTOR | CDSDP_SETUP_MERGE_CLIQUES)) return CDSDP_ERR_ARG;
    const bool cache_factor = !(flags & CDSDP_SETUP_NO_FACTOR);
    const bool merge = (flags & CDSDP_SETUP_MERGE_CLIQUES) != 0;
    if (scale_passes >= 0) {  // the factors read the triplets before the setup validates them
        if (n < 1 || m < 0 || nnzA < 0 || nnzC < 0) return CDSDP_ERR_ARG;
        if ((nnzA > 0 && (!A_con || !A_row || !A_col || !A_val)) || (m > 0 && !b) ||
            (nnzC > 0 && (!C_row || !C_col || !C_val)))
            return CDSDP_ERR_ARG;
        for (long long k = 0; k < nnzA; ++k)
            if (A_con[k] < 0 || A_con[k] >= m || A_row[k] < 0 || A_row[k] >= n || A_col[k] < 0 || A_col[k] >= n)
                return CDSDP_ERR_ARG;
        for (long long k = 0; k < nnzC; ++k)
            if (C_row[k] < 0 || C_row[k] >= n || C_col[k] < 0 || C_col[k] >= n) return CDSDP_ERR_ARG;
    }
    cdsdp* h = new (std::nothrow) cdsdp();
    if (!h) return CDSDP_ERR_NOMEM;
    int st;
    try {
        if (scale_passes < 0) {
            st = cdsdp_impl::build_host_problem(n, m, nnzA, A_con, A_row, A_col, A_val, b, nnzC, C_row, C_col,
                                                C_val, nnzP, P_row, P_col, h->hp, cache_factor, merge);
        } else {
            std::vector<double> d, e;
            double tau = 1.0, sigma = 1.0;
            cdsdp_impl::scaling_factors(n, m, nnzA, A_con, A_row, A_col, A_val, b, nnzC, C_row, C_col, C_val,
                                        scale_passes, d, e, tau, sigma);
            // tau and sigma per vertex and per constraint: the problem's, or in a
            // batch those of each SDP alone, 1 / ||E b_j|| and 1 / ||D C_j D||_F
            // (the equilibration passes act within each SDP already)
            const int nb = count > 0 ? count : 1;
            std::vector<double> tb(nb, tau), sb(nb, sigma), tv(n), sv(n), tr(m), sr(m);
            std::vector<int> sdp_of_v(n, 0), sdp_of_r(m, 0);
            if (count > 0) {
                for (int j = 0, vo = 0, mo = 0; j < count; vo += sdp_n[j], mo += sdp_m[j], ++j) {
                    for (int v = vo; v < vo + sdp_n[j]; ++v) sdp_of_v[v] = j;
                    for (int i = mo; i < mo + sdp_m[j]; ++i) sdp_of_r[i] = j;
                }
                std::vector<double> nbj(count, 0.0), ncj(count, 0.0);
                for (int i = 0; i < m; ++i) nbj[sdp_of_r[i]] += (e[i] * b[i]) * (e[i] * b[i]);
                for (long long k = 0; k < nnzC; ++k) {
                    const double v = d[C_row[k]] * d[C_col[k]] * C_val[k];
                    ncj[sdp_of_v[C_row[k]]] += (C_row[k] == C_col[k] ? 1.0 : 2.0) * v * v;
                }
                for (int j = 0; j < count; ++j) {
                    const double a = std::sqrt(nbj[j]), c = std::sqrt(ncj[j]);
                    tb[j] = a > 0.0 ? 1.0 / a : 1.0;
                    sb[j] = c > 0.0 ? 1.0 / c : 1.0;
                }
            }
            for (int v = 0; v < n; ++v) { tv[v] = tb[sdp_of_v[v]]; sv[v] = sb[sdp_of_v[v]]; }
            for (int i = 0; i < m; ++i) { tr[i] = tb[sdp_of_r[i]]; sr[i] = sb[sdp_of_r[i]]; }
            std::vector<double> av(nnzA), bv(m), cv(nnzC);
            for (long long k = 0; k < nnzA; ++k) av[k] = e[A_con[k]] * d[A_row[k]] * d[A_col[k]] * A_val[k];
            for (int i = 0; i < m; ++i) bv[i] = tr[i] * e[i] * b[i];
            for (long long k = 0; k < nnzC; ++k) cv[k] = sv[C_row[k]] * d[C_row[k]] * d[C_col[k]] * C_val[k];
            st = cdsdp_impl::build_host_problem(n, m, nnzA, A_con, A_row, A_col, av.data(), bv.data(), nnzC, C_row,
                                                C_col, cv.data(), nnzP, P_row, P_col, h->hp, cache_factor, merge);
            if (st == CDSDP_SOLVED) {
                h->hp.scaled = true;
                h->hp.sc_d = std::move(d);
                h->hp.sc_e = std::move(e);
                h->hp.sc_tau = tb[0];
                h->hp.sc_sigma = sb[0];
                h->hp.sc_tau_v = std::move(tv);
                h->hp.sc_sigma_v = std::move(sv);
                h->hp.sc_tau_r = std::move(tr);
                h->hp.sc_sigma_r = std::move(sr);
                h->hp.sc_tau_b = std::move(tb);
                h->hp.sc_sigma_b = std::move(sb);
            }
        }
    } catch (const std::exception&) {  // allocation or thread creation failed
        st = CDSDP_ERR_NOMEM;
    }
    if (st != CDSDP_SOLVED) { delete h; return st; }
    *out = h;
    return CDSDP_SOLVED;
}

}  // namespace

int cdsdp_setup(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                const double* b, long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                long long nnzP, const int* P_row, const int* P_col, cdsdp** out) {
    return setup_common(n, m, nnzA, A_con, A_row, A_col, A_val, b, nnzC, C_row, C_col, C_val, nnzP, P_row, P_col,
                        -1, 0u, out);
}

int cdsdp_setup_scaled(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col,
                       const double* A_val, const double* b, long long nnzC, const int* C_row, const int* C_col,
                       const double* C_val, long long nnzP, const int* P_row, const int* P_col, int scale_passes,
                       cdsdp** out) {
    if (out) *out = nullptr;
    if (scale_passes < 0) return CDSDP_ERR_ARG;
    return setup_common(n, m, nnzA, A_con, A_row, A_col, A_val, b, nnzC, C_row, C_col, C_val, nnzP, P_row, P_col,
                        scale_passes, 0u, out);
}

int cdsdp_setup_flags(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col,
                      const double* A_val, const double* b, long long nnzC, const int* C_row, const int* C_col,
                      const double* C_val, long long nnzP, const int* P_row, const int* P_col, int scale_passes,
                      unsigned flags, cdsdp** out) {
    return setup_common(n, m, nnzA, A_con, A_row, A_col, A_val, b, nnzC, C_row, C_col, C_val, nnzP, P_row, P_col,
                        scale_passes, flags, out);
}

int cdsdp_setup_batch(int count, const int* n, const int* m, const long long* nnzA, const int* A_con,
                      const int* A_row, const int* A_col, const double* A_val, const double* b,
                      const long long* nnzC, const int* C_row, const int* C_col, const double* C_val,
                      const long long* nnzP, const int* P_row, const int* P_col, int scale_passes, unsigned flags,
                      cdsdp** out) {
    if (!out) return CDSDP_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !n || !m || !nnzA || !nnzC) return CDSDP_ERR_ARG;
    long long N = 0, M = 0, tA = 0, tC = 0, tP = 0;
    for (int j = 0; j < count; ++j) {
        if (n[j] < 1 || m[j] < 1 || nnzA[j] < 0 || nnzC[j] < 0 || (nnzP && nnzP[j] < 0)) return CDSDP_ERR_ARG;
        N += n[j];
        M += m[j];
        tA += nnzA[j];
        tC += nnzC[j];
        if (nnzP) tP += nnzP[j];
    }
    if (N > 2000000000LL || M > 2000000000LL) return CDSDP_ERR_UNSUPPORTED;
    if ((tA > 0 && (!A_con || !A_row || !A_col || !A_val)) || !b || (tC > 0 && (!C_row || !C_col || !C_val)) ||
        (tP > 0 && (!P_row || !P_col)))
        return CDSDP_ERR_ARG;
    try {
        // the direct sum: problem j's vertices and constraints shifted past
        // those of problems 0..j-1; local indices are checked against n_j, m_j
        std::vector<int> ac(tA), ar(tA), acl(tA), cr(tC), cc(tC), pr(tP), pc(tP);
        long long ka = 0, kc = 0, kp = 0;
        int vo = 0, mo = 0;
        for (int j = 0; j < count; ++j) {
            for (long long q = 0; q < nnzA[j]; ++q, ++ka) {
                if (A_con[ka] < 0 || A_con[ka] >= m[j] || A_row[ka] < 0 || A_row[ka] >= n[j] || A_col[ka] < 0 ||
                    A_col[ka] >= n[j])
                    return CDSDP_ERR_ARG;
                ac[ka] = A_con[ka] + mo;
                ar[ka] = A_row[ka] + vo;
                acl[ka] = A_col[ka] + vo;
            }
            for (long long q = 0; q < nnzC[j]; ++q, ++kc) {
                if (C_row[kc] < 0 || C_row[kc] >= n[j] || C_col[kc] < 0 || C_col[kc] >= n[j]) return CDSDP_ERR_ARG;
                cr[kc] = C_row[kc] + vo;
                cc[kc] = C_col[kc] + vo;
            }
            for (long long q = 0; nnzP && q < nnzP[j]; ++q, ++kp) {
                if (P_row[kp] < 0 || P_row[kp] >= n[j] || P_col[kp] < 0 || P_col[kp] >= n[j]) return CDSDP_ERR_ARG;
                pr[kp] = P_row[kp] + vo;
                pc[kp] = P_col[kp] + vo;
            }
            vo += n[j];
            mo += m[j];
        }
        return setup_common((int)N, (int)M, tA, ac.data(), ar.data(), acl.data(), A_val, b, tC, cr.data(), cc.data(),
                            C_val, tP, pr.data(), pc.data(), scale_passes, flags, out, count, n, m);
    } catch (const std::exception&) {  // allocation failed
        return CDSDP_ERR_NOMEM;
    }
}

int cdsdp_scaling(const cdsdp* h, double* d, double* e, double* tau, double* sigma) {
    if (!h) return CDSDP_ERR_ARG;
    const HostProblem& hp = h->hp;
    if (d) {
        if (hp.scaled) std::copy(hp.sc_d.begin(), hp.sc_d.end(), d);
        else std::fill(d, d + hp.n, 1.0);
    }
    if (e) {
        if (hp.scaled) std::copy(hp.sc_e.begin(), hp.sc_e.end(), e);
        else std::fill(e, e + hp.m, 1.0);
    }
    if (tau) *tau = hp.sc_tau;
    if (sigma) *sigma = hp.sc_sigma;
    return CDSDP_SOLVED;
}

int cdsdp_scaling_batch(const cdsdp* h, int* count, double* tau, double* sigma) {
    if (!h) return CDSDP_ERR_ARG;
    const HostProblem& hp = h->hp;
    const int nb = hp.scaled ? (int)hp.sc_tau_b.size() : 1;
    if (count) *count = nb;
    for (int j = 0; j < nb; ++j) {
        if (tau) tau[j] = hp.scaled ? hp.sc_tau_b[j] : 1.0;
        if (sigma) sigma[j] = hp.scaled ? hp.sc_sigma_b[j] : 1.0;
    }
    return CDSDP_SOLVED;
}

int cdsdp_completion_sizes(const cdsdp* h, size_t* scratch_bytes, long long* w_elems, long long* w_offsets) {
    if (h && h->hp.merged) return CDSDP_ERR_UNSUPPORTED;
    if (!h) return CDSDP_ERR_ARG;
    try {
        return cdsdp_impl::completion_sizes(h->hp, scratch_bytes, w_elems, w_offsets);
    } catch (const std::exception&) {  // allocation or thread creation failed
        return CDSDP_ERR_NOMEM;
    }
}

int cdsdp_complete(cdsdp* h, const double* d_X, void* d_scratch, size_t scratch_bytes, double* d_W, double* logdet,
                   void* stream) {
    if (h && h->hp.merged) return CDSDP_ERR_UNSUPPORTED;
    if (!h) return CDSDP_ERR_ARG;
    try {
        return cdsdp_impl::completion_run(h->hp, d_X, d_scratch, scratch_bytes, d_W, logdet, stream, &h->err,
                                          &h->cmp_graph);
    } catch (const std::exception&) {  // allocation or thread creation failed
        return CDSDP_ERR_NOMEM;
    }
}

int cdsdp_info(const cdsdp* h, cdsdp_info_t* info) {
    if (!h || !info) return CDSDP_ERR_ARG;
    const HostProblem& hp = h->hp;
    info->n = hp.n;
    info->m = hp.m;
    info->p = (int)hp.cl_off.size() - 1;
    info->max_clique = hp.max_clique;
    info->nnz_pattern = (long long)hp.prow.size();
    info->n_d_lower = (long long)hp.gmap.size();
    info->nnz_A = (long long)hp.a_col.size();
    info->n_fill = hp.nfill;
    info->chordal = hp.chordal ? 1 : 0;
    info->diag_factor = hp.diag_factor ? 1 : 0;
    info->upload_bytes = (long long)make_layout(hp, 1).const_end;
    info->ncomp = hp.ncomp;
    info->cached_factor = hp.cached_factor ? 1 : 0;
    return CDSDP_SOLVED;
}

int cdsdp_cliques(const cdsdp* h, int* offsets, int* vertices) {
    if (!h || !offsets || !vertices) return CDSDP_ERR_ARG;
    std::copy(h->hp.cl_off.begin(), h->hp.cl_off.end(), offsets);
    std::copy(h->hp.cl_vert.begin(), h->hp.cl_vert.end(), vertices);
    return CDSDP_SOLVED;
}

int cdsdp_pattern(const cdsdp* h, int* rows, int* cols) {
    if (!h || !rows || !cols) return CDSDP_ERR_ARG;
    std::copy(h->hp.prow.begin(), h->hp.prow.end(), rows);
    std::copy(h->hp.pcol.begin(), h->hp.pcol.end(), cols);
    return CDSDP_SOLVED;
}

int cdsdp_components(const cdsdp* h, int* vertex_comp, int* constraint_comp) {
    if (!h) return CDSDP_ERR_ARG;
    if (vertex_comp) std::copy(h->hp.comp_of_vertex.begin(), h->hp.comp_of_vertex.end(), vertex_comp);
    if (constraint_comp) std::copy(h->hp.comp_of_row.begin(), h->hp.comp_of_row.end(), constraint_comp);
    return CDSDP_SOLVED;
}

int cdsdp_component_results(cdsdp* h, void* stream, int* iters, int* status, double* res) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->ws || h->last_form < 0) return CDSDP_ERR_STATE;
    const int nc = h->hp.ncomp;
    cudaStream_t st = (cudaStream_t)stream;
    const Dev& d = h->dev;
    if (h->last_comp_mode) {
        if (iters) CK(cudaMemcpyAsync(iters, d.comp_iter, nc * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (status) CK(cudaMemcpyAsync(status, d.comp_status, nc * sizeof(int), cudaMemcpyDeviceToHost, st));
        if (res) CK(cudaMemcpyAsync(res, d.comp_res, (size_t)nc * HIST_COLS * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return CDSDP_SOLVED;
    }
    // one test over the whole problem: every component shares it
    double last[HIST_COLS] = {0};
    if (res && h->last_iters > 0) {
        CK(cudaMemcpyAsync(last, d.hist + (size_t)(h->last_iters - 1) * HIST_COLS, sizeof(last),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    for (int c = 0; c < nc; ++c) {
        if (iters) iters[c] = h->last_iters;
        if (status) status[c] = h->last_status;
        if (res) std::copy(last, last + HIST_COLS, res + (size_t)c * HIST_COLS);
    }
    return CDSDP_SOLVED;
}

int cdsdp_workspace_bytes(const cdsdp* h, int max_iter, size_t* bytes) {
    if (!h || !bytes || max_iter < 1) return CDSDP_ERR_ARG;
    *bytes = make_layout(h->hp, max_iter).ws_end;
    return CDSDP_SOLVED;
}

int cdsdp_bind(cdsdp* h, void* d_workspace, size_t bytes, int max_iter, void* stream) {
    if (!h || !d_workspace || max_iter < 1) return CDSDP_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) return CDSDP_ERR_ARG;
    if (h->hp.max_clique > cdsdp_large::kMaxLargeOrder) return CDSDP_ERR_UNSUPPORTED;
    Layout L = make_layout(h->hp, max_iter);
    if (bytes < L.ws_end) return CDSDP_ERR_NOMEM;
    drop_graph(h);
    h->L = L;
    h->ws = (unsigned char*)d_workspace;
    h->ws_bytes = bytes;
    h->ws_max_iter = max_iter;
    try {
        build_image(h);
    } catch (const std::exception&) {  // allocation or thread creation failed
        h->ws = nullptr;
        return CDSDP_ERR_NOMEM;
    }
    make_dev(h);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h->ws, h->image.data(), h->image.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    // large cliques: tensor maps of the dense buffers (they encode the
    // workspace address), tables, and zero padding of the W buffers
    std::vector<int> list;
    std::vector<long long> poff;
    for (size_t k = 0; k + 1 < h->hp.cl_off.size(); ++k)
        if (h->hp.cl_off[k + 1] - h->hp.cl_off[k] >= cdsdp_large::kLargeFrom) {
            list.push_back((int)k);
            poff.push_back(h->hp.pk_off[k]);
        }
    {
        double work[kNumClasses] = {0};
        for (size_t k = 0; k + 1 < h->hp.cl_off.size(); ++k) {
            const double sk = h->hp.cl_off[k + 1] - h->hp.cl_off[k];
            const int c = class_of((int)sk);
            if (c >= 0) work[c] += sk * sk * sk;
        }
        for (int c = 0; c < kNumClasses; ++c) h->cls_order[c] = c;
        std::stable_sort(h->cls_order, h->cls_order + kNumClasses, [&](int a, int b) { return work[a] > work[b]; });
        if (!h->side[0] && h->hp.ncomp > 1) {
            for (int i = 0; i < 4; ++i) {
                CK(cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming));
            }
            CK(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        }
    }
    h->ns = cdsdp_large::ns_layout(large_sizes(h->hp));
    if (h->ns.nb > 0) {
        std::vector<unsigned char> img;
        unsigned char* base = h->ws + L.ns_off;
        if (!cdsdp_large::ns_tables(h->ns, base, poff, list, img)) {
            h->err = "tensor-map encoder unavailable or refused a map";
            h->ws = nullptr;
            return CDSDP_ERR_CUDA;
        }
        CK(cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(base + h->ns.o_buf[2 * cdsdp_large::BUF_W], 0,
                           2 * (size_t)h->ns.elems * sizeof(float), st));
        CK(cudaStreamSynchronize(st));
    }
    return CDSDP_SOLVED;
}

int cdsdp_solve(cdsdp* h, int form, const cdsdp_opts* opts, void* stream, double* X, double* y, double* Z,
                double* hist, int* iters, double* cert) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->ws) return CDSDP_ERR_STATE;
    if (form < 0 || form > 2) return CDSDP_ERR_ARG;
    cdsdp_opts o;
    if (opts) o = *opts; else cdsdp_default_opts(&o);
    int rc = check_opts(h, o);
    if (rc != CDSDP_SOLVED) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (form == 2 && o.linear_solver == 1) return CDSDP_ERR_UNSUPPORTED;
    if (!h->hp.cached_factor && (form == 2 || o.linear_solver == 0)) return CDSDP_ERR_UNSUPPORTED;
    if (form == 2 && (rc = ensure_hsde(h, st)) != CDSDP_SOLVED) return rc;
    Dev& d = h->dev;
    d.max_iter = o.max_iter;
    // threads per constraint row of the A-row kernels, and the row grid
    h->TPR = o.row_threads ? o.row_threads : h->TPR_auto;
    {
        const int TP = std::max(h->TPR, h->TPRM);
        h->GR = std::max(1, std::min(NBLK_R, (d.m + RTHREADS / TP - 1) / (RTHREADS / TP)));
    }
    d.comp_mode = (h->hp.ncomp > 1 && o.component_stop && o.linear_solver == 0) ? 1 : 0;
    // Algorithm 3: one embedding per component in component mode, else one over the whole problem
    const bool hs_comp = form == 2 && d.comp_mode;
    d.zhx = (const double*)(h->ws + (hs_comp ? h->L.zhx_c : h->L.zhx));
    d.zhy = (const double*)(h->ws + (hs_comp ? h->L.zhy_c : h->L.zhy));
    d.azhx = (const double*)(h->ws + (hs_comp ? h->L.azhx_c : h->L.azhx));
    d.cg_tol = o.cg_tol;
    d.cg_max = o.cg_max_steps;
    h->x_split = h->ns.nb > 0 || (o.x_update == 0 ? h->x_split_auto : o.x_update == 2);
    // zero the state (clique vectors, iterates, partials, history)
    CK(cudaMemsetAsync(h->ws + h->L.const_end, 0, h->L.total - h->L.const_end, st));
    k_init<<<1, 256, 0, st>>>(d, form, o.rho);
    CK(cudaGetLastError());
    h->last_profiled = false;
    if (o.profile) {
        // 4 events per iteration: iteration start, projection start/end, iteration end
        const size_t need = (size_t)4 * o.max_iter;
        while (h->ev.size() < need) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            h->ev.push_back(e);
        }
        const size_t need_cls = (size_t)(2 * kNumClasses + 2) * o.max_iter;
        while (h->cls_evs.size() < need_cls) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            h->cls_evs.push_back(e);
        }
        int ctl[CTL_WORDS];
        int launched = 0;
        for (int it = 0; it < o.max_iter; ++it) {
            CK(cudaEventRecord(h->ev[4 * it], st));
            h->cls_ev = h->cls_evs.data() + (size_t)(2 * kNumClasses + 2) * it;
            const cudaError_t le =
                launch_iteration_any(h, form, o, st, 0, cudaGraphConditionalHandle{}, h->ev[4 * it + 1], h->ev[4 * it + 2]);
            h->cls_ev = nullptr;
            CK(le);
            CK(cudaEventRecord(h->ev[4 * it + 3], st));
            ++launched;
            if ((it + 1) % o.check_every == 0 || it + 1 == o.max_iter) {
                CK(cudaMemcpyAsync(ctl, d.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (ctl[CTL_DONE]) break;
            }
        }
        CK(cudaStreamSynchronize(st));
        CK(cudaMemcpyAsync(ctl, d.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const int ran = std::min(launched, ctl[CTL_ITER]);
        h->prof_proj_ms = h->prof_iter_ms = 0.0;
        for (int c = 0; c < kNumClasses; ++c) {
            h->prof_cls_ms[c] = 0.0;
            h->prof_cls_n[c] = 0;
        }
        h->prof_large_ms = 0.0;
        h->prof_large_n = 0;
        for (int it = 0; it < ran; ++it) {
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, h->ev[4 * it + 1], h->ev[4 * it + 2]));
            CK(cudaEventElapsedTime(&b, h->ev[4 * it], h->ev[4 * it + 3]));
            h->prof_proj_ms += a;
            h->prof_iter_ms += b;
            for (int c = 0; c < kNumClasses; ++c) {
                if (h->cls_off[c + 1] <= h->cls_off[c]) continue;
                const cudaEvent_t* pe = h->cls_evs.data() + (size_t)(2 * kNumClasses + 2) * it + 2 * c;
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, pe[0], pe[1]));
                h->prof_cls_ms[c] += t;
                h->prof_cls_n[c] += 1;
            }
            if (h->ns.nb > 0) {
                const cudaEvent_t* pe = h->cls_evs.data() + (size_t)(2 * kNumClasses + 2) * it + 2 * kNumClasses;
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, pe[0], pe[1]));
                h->prof_large_ms += t;
                h->prof_large_n += 1;
            }
        }
        h->prof_launches = ran;
        h->last_profiled = true;
    } else if (o.use_graph) {
        if (!h->gexec || h->g_form != form || !same_opts(h->g_opts, o)) {
            rc = build_graph(h, form, o);
            if (rc != CDSDP_SOLVED) return rc;
        }
        CK(cudaGraphLaunch(h->gexec, st));
    } else {
        int ctl[CTL_WORDS];
        for (int it = 0; it < o.max_iter; ++it) {
            CK(launch_iteration_any(h, form, o, st, 0, cudaGraphConditionalHandle{}));
            if ((it + 1) % o.check_every == 0 || it + 1 == o.max_iter) {
                CK(cudaMemcpyAsync(ctl, d.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (ctl[CTL_DONE]) break;
            }
        }
        h->g_opts = o;
    }
    int ctl[CTL_WORDS];
    CK(cudaMemcpyAsync(ctl, d.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->g_opts = o;
    h->last_form = form;
    h->last_iters = ctl[CTL_ITER];
    h->last_status = ctl[CTL_STATUS];
    h->last_comp_mode = d.comp_mode;
    if (iters) *iters = h->last_iters;
    if (h->ns.nb > 0) {  // a bounded wait inside the tensor-core products that ran out
        int nerr = 0;
        unsigned char* ep = h->ws + h->L.ns_off + h->ns.o_err;
        CK(cudaMemcpyAsync(&nerr, ep, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (nerr) {
            CK(cudaMemsetAsync(ep, 0, sizeof(int), st));
            h->err = "a bounded wait in the tensor-core product kernel ran out";
            return CDSDP_ERR_TIMEOUT;
        }
    }
    rc = copy_results(h, st, X, y, Z, hist, cert);
    if (rc != CDSDP_SOLVED) return rc;
    return h->last_status;
}

int cdsdp_results(cdsdp* h, void* stream, double* X, double* y, double* Z, double* hist, double* cert) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->ws || h->last_form < 0) return CDSDP_ERR_STATE;
    return copy_results(h, (cudaStream_t)stream, X, y, Z, hist, cert);
}

int cdsdp_autotune(cdsdp* h, int form, const cdsdp_opts* opts, int iters, void* stream, cdsdp_opts* tuned,
                   double* ms_per_iter, int* n_cand) {
    if (!h || !tuned || iters < 1) return CDSDP_ERR_ARG;
    if (!h->ws) return CDSDP_ERR_STATE;
    if (form < 0 || form > 2) return CDSDP_ERR_ARG;
    cdsdp_opts base;
    if (opts) base = *opts; else cdsdp_default_opts(&base);
    if (!h->hp.cached_factor && (form == 2 || base.linear_solver == 0)) return CDSDP_ERR_UNSUPPORTED;
    base.eps = 0.0;  // fixed number of iterations
    base.max_iter = std::min(iters, h->ws_max_iter);
    base.profile = 0;
    // candidate schedules: x-update placement (Algorithm 1), warps per block of
    // the warp-per-clique projections, cold-restart interval of the eigensolver
    std::vector<cdsdp_opts> cand;
    const int xs[2] = {2, 1}, wd[3] = {1, 2, 4}, rs[2] = {16, 64}, ps[2] = {4, 1};
    for (int xi = 0; xi < (form == 0 ? 2 : 1); ++xi)
        for (int wi = 0; wi < 3; ++wi)
            for (int ri = 0; ri < (base.warm_start > 0 ? 2 : 1); ++ri)
                for (int pi = 0; pi < 2; ++pi) {
                    cdsdp_opts o = base;
                    o.x_update = xs[xi];
                    o.proj_warps_div = wd[wi];
                    if (base.warm_start > 0) o.warm_start = rs[ri];
                    o.proj_streams = ps[pi];
                    cand.push_back(o);
                }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int ibest = 0, rc = CDSDP_SOLVED;
    // then, from the fastest so far: the other thread-block projection kernel,
    // and 64, 128 and 256 threads per constraint row
    const size_t n_grid = cand.size();
    const int rt[3] = {64, 128, 256};
    for (size_t i = 0; i < n_grid + 4 && rc >= 0; ++i) {
        if (i == n_grid) {
            cdsdp_opts o = cand[ibest];
            o.proj_cta_kernel = 1 - o.proj_cta_kernel;
            cand.push_back(o);
        } else if (i > n_grid) {
            cdsdp_opts o = cand[ibest];
            o.row_threads = rt[i - n_grid - 1];
            cand.push_back(o);
        }
        rc = cdsdp_solve(h, form, &cand[i], stream, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);  // warm-up
        if (rc < 0) break;
        cudaEventRecord(e0, st);
        rc = cdsdp_solve(h, form, &cand[i], stream, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        cudaEventRecord(e1, st);
        if (rc < 0) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / std::max(1, h->last_iters);
        if (ms_per_iter) ms_per_iter[i] = per;
        if (per < best) { best = per; ibest = (int)i; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc < 0) return rc;
    *tuned = opts ? *opts : cand[0];
    if (!opts) cdsdp_default_opts(tuned);
    tuned->x_update = cand[ibest].x_update;
    tuned->proj_warps_div = cand[ibest].proj_warps_div;
    tuned->warm_start = cand[ibest].warm_start;
    tuned->proj_streams = cand[ibest].proj_streams;
    tuned->proj_cta_kernel = cand[ibest].proj_cta_kernel;
    tuned->row_threads = cand[ibest].row_threads;
    if (n_cand) *n_cand = (int)cand.size();
    return CDSDP_SOLVED;
}

int cdsdp_profile_orders(const cdsdp* h, int* orders, double* ms, int* launches, int* cliques, double* nominal_flops) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->last_profiled) return CDSDP_ERR_STATE;
    for (int c = 0; c < kNumClasses; ++c) {
        if (orders) orders[c] = kProjClasses[c];
        if (ms) ms[c] = h->prof_cls_ms[c];
        if (launches) launches[c] = h->prof_cls_n[c];
        if (cliques) cliques[c] = h->cls_off[c + 1] - h->cls_off[c];
        if (nominal_flops) nominal_flops[c] = 0.0;
    }
    if (nominal_flops) {
        const size_t p = h->hp.cl_off.size() - 1;
        for (size_t k = 0; k < p; ++k) {
            const double s = double(h->hp.cl_off[k + 1] - h->hp.cl_off[k]);
            const int c = class_of(int(s));
            if (c >= 0) nominal_flops[c] += 10.0 * s * s * s;
        }
    }
    return CDSDP_SOLVED;
}

int cdsdp_profile_large(const cdsdp* h, double* ms, int* launches, int* cliques, double* nominal_flops,
                        double* tensor_flops) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->last_profiled) return CDSDP_ERR_STATE;
    if (ms) *ms = h->prof_large_ms;
    if (launches) *launches = h->prof_large_n;
    if (cliques) *cliques = h->ns.nb;
    double nom = 0.0, ten = 0.0;
    const int products = 3 * cdsdp_large::kPhase1 + 2 * cdsdp_large::kPhase2 + 1;
    for (const auto& b : h->ns.blocks) {
        nom += 10.0 * double(b.s) * b.s * b.s;
        const double T = b.S / cdsdp_large::kTile;
        ten += products * (T * (T + 1) / 2) * 3.0 * 2.0 * cdsdp_large::kTile * cdsdp_large::kTile * double(b.S);
    }
    if (nominal_flops) *nominal_flops = nom;
    if (tensor_flops) *tensor_flops = ten;
    return CDSDP_SOLVED;
}

int cdsdp_profile(const cdsdp* h, double* proj_ms, int* proj_launches, double* iter_ms) {
    if (!h) return CDSDP_ERR_ARG;
    if (!h->last_profiled) return CDSDP_ERR_STATE;
    if (proj_ms) *proj_ms = h->prof_proj_ms;
    if (proj_launches) *proj_launches = h->prof_launches;
    if (iter_ms) *iter_ms = h->prof_iter_ms;
    return CDSDP_SOLVED;
}

int cdsdp_free(cdsdp* h) {
    if (!h) return CDSDP_ERR_ARG;
    drop_graph(h);
    cdsdp_impl::completion_release(h->cmp_graph);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->cls_evs) cudaEventDestroy(e);
    for (int i = 0; i < 4; ++i) {
        if (h->side[i]) cudaStreamDestroy(h->side[i]);
        if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    delete h;
    return CDSDP_SOLVED;
}

const char* cdsdp_strerror(int s) {
    switch (s) {
        case CDSDP_SOLVED: return "solved";
        case CDSDP_MAX_ITER: return "maximum number of iterations reached";
        case CDSDP_PRIMAL_INFEASIBLE: return "primal infeasible (certificate returned)";
        case CDSDP_DUAL_INFEASIBLE: return "dual infeasible (certificate returned)";
        case CDSDP_NOT_PD: return "a clique block is not positive definite (no completion)";
        case CDSDP_ERR_ARG: return "invalid argument";
        case CDSDP_ERR_RANK: return "A is not full row rank (factorisation failed)";
        case CDSDP_ERR_CUDA: return "CUDA runtime error";
        case CDSDP_ERR_NOMEM: return "out of memory or workspace too small";
        case CDSDP_ERR_TIMEOUT: return "bounded device wait timed out";
        case CDSDP_ERR_NUMERIC: return "NaN or Inf in the iteration";
        case CDSDP_ERR_STATE: return "call out of order";
        case CDSDP_ERR_UNSUPPORTED: return "size or option not supported by the library";
        default: return "unknown status";
    }
}

int cdsdp_psd_project(int p, const int* d_off, const int* d_size, int max_size, const void* d_W, void* d_X, void* d_eig,
                      const int* d_voff, void* d_V, const int* d_vvoff, int precision, int max_sweeps, void* stream) {
    cdsdp* h = nullptr;
    if (p < 0 || max_size < 1 || max_sweeps < 1) return p == 0 ? CDSDP_SOLVED : CDSDP_ERR_ARG;
    if (max_size > (precision == CDSDP_FP64 ? kMaxOrderF64 : kMaxOrderF32)) return CDSDP_ERR_UNSUPPORTED;
    if (p == 0) return CDSDP_SOLVED;
    if (!d_off || !d_size || !d_W || !d_X) return CDSDP_ERR_ARG;
    if ((d_eig && !d_voff) || (d_V && !d_vvoff)) return CDSDP_ERR_ARG;
    if ((d_eig || d_V) && max_size > kMaxWarpOrder) return CDSDP_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int c = class_of(max_size);
    cudaError_t e;
    if (precision == CDSDP_FP64)
        e = launch_proj_standalone_f64(c, p, d_off, d_size, d_W, d_X, d_eig, d_voff, d_V, d_vvoff, 2.3e-16, max_sweeps, st);
    else if (precision == CDSDP_FP32_PROJECTION)
        e = launch_proj_standalone_f32(c, p, d_off, d_size, d_W, d_X, d_eig, d_voff, d_V, d_vvoff, 1.2e-7, max_sweeps, st);
    else
        return CDSDP_ERR_ARG;
    CK(e);
    CK(cudaGetLastError());
    return CDSDP_SOLVED;
}


int cdsdp_grad_workspace_bytes(const cdsdp* h, int iters, int ckpt_every, int precision, size_t* bytes) {
    if (!h || !bytes || iters < 1 || ckpt_every < 1) return CDSDP_ERR_ARG;
    if (!h->ws) return CDSDP_ERR_STATE;
    *bytes = make_grad_layout(h->dev, iters, ckpt_every, precision != CDSDP_FP64).total;
    return CDSDP_SOLVED;
}

int cdsdp_unrolled_forward(cdsdp* h, const cdsdp_opts* opts, int iters, int ckpt_every, const double* d_c,
                           const double* d_b, void* d_gws, size_t gws_bytes, double* d_x, void* stream) {
    if (!h || !d_c || !d_b || !d_gws || !d_x) return CDSDP_ERR_ARG;
    const cdsdp_opts o = unrolled_opts(opts);
    h->x_split = h->ns.nb > 0 || (o.x_update == 0 ? h->x_split_auto : o.x_update == 2);
    int rc = check_unrolled(h, o, iters, ckpt_every);
    if (rc != CDSDP_SOLVED) return rc;
    const bool fp32 = o.precision != CDSDP_FP64;
    const GradLayout G = make_grad_layout(h->dev, iters, ckpt_every, fp32);
    if (gws_bytes < G.total) return CDSDP_ERR_NOMEM;
    if (reinterpret_cast<uintptr_t>(d_gws) % kAlign) return CDSDP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* g = (unsigned char*)d_gws;
    Dev dd = h->dev;
    dd.c = d_c;
    dd.b = d_b;
    dd.max_iter = ckpt_every;
    dd.comp_mode = 0;
    const size_t ts = fp32 ? 4 : 8, nd = dd.nd;
    CK(cudaMemsetAsync(h->ws + h->L.const_end, 0, h->L.total - h->L.const_end, st));
    for (int sg = 0; sg < G.nseg; ++sg) {
        unsigned char* ck = g + G.ckpt + (size_t)sg * 2 * nd * ts;
        CK(cudaMemcpyAsync(ck, dd.ck0, nd * ts, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ck + nd * ts, dd.ck1, nd * ts, cudaMemcpyDeviceToDevice, st));
        const int len = std::min(ckpt_every, iters - sg * ckpt_every);
        rc = run_segment(h, dd, o, len, st);
        if (rc != CDSDP_SOLVED) return rc;
    }
    CK(cudaMemcpyAsync(d_x, dd.x, (size_t)dd.NE * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return CDSDP_SOLVED;
}

int cdsdp_unrolled_backward(cdsdp* h, const cdsdp_opts* opts, int iters, int ckpt_every, const double* d_c,
                            const double* d_b, void* d_gws, size_t gws_bytes, const double* d_xbar, double* d_cbar,
                            double* d_bbar, void* stream) {
    if (!h || !d_c || !d_b || !d_gws || !d_xbar || !d_cbar || !d_bbar) return CDSDP_ERR_ARG;
    const cdsdp_opts o = unrolled_opts(opts);
    h->x_split = h->ns.nb > 0 || (o.x_update == 0 ? h->x_split_auto : o.x_update == 2);
    int rc = check_unrolled(h, o, iters, ckpt_every);
    if (rc != CDSDP_SOLVED) return rc;
    const bool fp32 = o.precision != CDSDP_FP64;
    const GradLayout G = make_grad_layout(h->dev, iters, ckpt_every, fp32);
    if (gws_bytes < G.total) return CDSDP_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* g = (unsigned char*)d_gws;
    Dev dd = h->dev;
    dd.c = d_c;
    dd.b = d_b;
    dd.max_iter = ckpt_every;
    dd.wstore = g + G.wstore;
    dd.wstore_count = ckpt_every;
    dd.comp_mode = 0;
    const size_t ts = fp32 ? 4 : 8, nd = dd.nd;
    double* xkbar = (double*)(g + G.xkbar);
    double* lambar = (double*)(g + G.lambar);
    double* hxbar = (double*)(g + G.hxbar);
    double* lamprev = (double*)(g + G.lamprev);
    double* xbar = (double*)(g + G.xbar);
    double* u = (double*)(g + G.u);
    double* sbar = (double*)(g + G.sbar);
    double* ybar = (double*)(g + G.ybar);
    double* rbar = (double*)(g + G.rbar);
    CK(cudaMemsetAsync(xkbar, 0, nd * 8, st));
    CK(cudaMemsetAsync(lambar, 0, nd * 8, st));
    CK(cudaMemsetAsync(d_cbar, 0, (size_t)dd.NE * 8, st));
    CK(cudaMemsetAsync(d_bbar, 0, (size_t)dd.m * 8, st));
    const int* bl = (const int*)(h->ws + h->L.blist);
    const int GE = std::max(1, std::min(NBLK_E, (dd.NE + ETHREADS - 1) / ETHREADS));
    const int GR = std::max(1, std::min(NBLK_R, (dd.m + 7) / 8));
    const int GN = std::max(1, std::min(NBLK_E, (dd.nd + ETHREADS - 1) / ETHREADS));
    GradArgs ga;
    ga.xkbar = xkbar; ga.lambar = lambar; ga.hxbar = hxbar; ga.lamprev = lamprev;
    ga.rho = o.rho; ga.tolrel = 0.0; ga.max_sweeps = o.jacobi_max_sweeps;
    for (int sg = G.nseg - 1; sg >= 0; --sg) {
        unsigned char* ck = g + G.ckpt + (size_t)sg * 2 * nd * ts;
        CK(cudaMemsetAsync(h->ws + h->L.const_end, 0, h->L.total - h->L.const_end, st));
        CK(cudaMemcpyAsync(dd.ck0, ck, nd * ts, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(dd.ck1, ck + nd * ts, nd * ts, cudaMemcpyDeviceToDevice, st));
        const int len = std::min(ckpt_every, iters - sg * ckpt_every);
        rc = run_segment(h, dd, o, len, st);  // replay, recording W of every iteration
        if (rc != CDSDP_SOLVED) return rc;
        for (int n = len - 1; n >= 0; --n) {
            ga.slot = n;
            for (int c = 0; c < kNumClasses; ++c) {
                const int nl = h->cls_off[c + 1] - h->cls_off[c];
                if (nl <= 0) continue;
                CK(launch_bwd_proj(fp32, c, dd, bl + h->cls_off[c], nl, ga, st));
            }
            const bool last = (sg * ckpt_every + n == iters - 1);
            k_bwd_scatter<<<GE, ETHREADS, 0, st>>>(dd, hxbar, last ? d_xbar : nullptr, xbar, u);
            k_bwd_ybar<<<GR, RTHREADS, 0, st>>>(dd, u, ybar);
            k_bwd_rbar<<<GR, RTHREADS, 0, st>>>(dd, ybar, rbar, d_bbar);
            k_bwd_tbar<<<GE, ETHREADS, 0, st>>>(dd, xbar, rbar, sbar, d_cbar, o.rho);
            k_bwd_state<<<GN, ETHREADS, 0, st>>>(dd, sbar, lamprev, xkbar, lambar, o.rho);
            CK(cudaGetLastError());
        }
    }
    return CDSDP_SOLVED;
}

}  // extern "C"
