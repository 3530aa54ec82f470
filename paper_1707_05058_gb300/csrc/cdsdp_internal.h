// Internal declarations shared by the host setup (setup.cpp) and the CUDA
// solver (solver.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <new>
#include <type_traits>
#include <utility>
#include <string>
#include <vector>

#include "../../include/cdsdp.h"

namespace cdsdp_impl {

// Allocator whose value-initialisation leaves trivially constructible
// elements uninitialised, so that resizing the large host arrays does not
// zero gigabytes on one thread before the threads fill them.
template <typename T>
struct DefaultInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = DefaultInitAlloc<U>;
    };
    DefaultInitAlloc() noexcept = default;
    template <typename U>
    DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
    template <typename U>
    void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new (static_cast<void*>(p)) U;
    }
    template <typename U, typename... Args>
    void construct(U* p, Args&&... args) {
        ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
    }
};
template <typename T>
using BigVec = std::vector<T, DefaultInitAlloc<T>>;

// Everything the data-preprocessing step of Algorithms 1-3 produces, on the host.
struct HostProblem {
    int n = 0, m = 0;
    // extended pattern E*, lower entries (row >= col), column-major order
    std::vector<int> prow, pcol, colptr;  // colptr[n+1] indexes prow/pcol
    // perfect elimination order of the extended pattern (vertex eliminated at
    // step k) and, per vertex, its neighbours eliminated after it (a clique),
    // ascending: lt_idx[lt_ptr[v] .. lt_ptr[v+1])
    std::vector<int> peo, lt_ptr, lt_idx;
    // maximal cliques, each ascending, list in lexicographic order
    std::vector<int> cl_off, cl_vert;
    int max_clique = 0;
    // lower-packed clique storage: clique k owns [pk_off[k], pk_off[k+1]);
    // entry (a, b), a >= b, of the |C_k| x |C_k| block sits at
    // pk_off[k] + b*(2s - b + 1)/2 + (a - b)
    std::vector<int> pk_off;
    BigVec<int> gmap;                 // packed position -> pattern entry (H_k)
    std::vector<int> sc_ptr;          // pattern entry -> packed positions (H^T)
    BigVec<int> sc_idx;
    std::vector<double> c, D;         // per pattern entry
    // A as CSR over (constraint, pattern entry), unweighted values
    std::vector<int> a_ptr;
    BigVec<int> a_col;
    BigVec<double> a_val;
    // A^T as CSR over (pattern entry, constraint)
    std::vector<int> at_ptr;
    BigVec<int> at_col;
    BigVec<double> at_val;
    std::vector<double> b;
    long long nfill = 0;
    bool chordal = false;
    bool merged = false;              // cliques merged (CDSDP_SETUP_MERGE_CLIQUES); the PEO lists are not rebuilt
    bool diag_factor = false;
    // Independent components (connected components of the extended pattern with
    // every constraint joining the vertices of its entries): a direct sum of
    // SDPs has one per summand.  A D^-1 A^T is block diagonal over them.
    int ncomp = 1;
    std::vector<int> comp_of_vertex, comp_of_entry, comp_of_clique, comp_of_row;  // [n], [NE], [p], [m]
    bool rows_contiguous = true;       // constraints of each component form one index range
    std::vector<int> lrow;             // [m] index of a constraint within its component
    std::vector<int> crow_ptr, crow_idx;  // constraints of each component (ascending)
    std::vector<int> ccl_ptr, ccl_idx;    // cliques of each component (ascending)
    std::vector<int> cent_ptr, cent_idx;  // pattern entries of each component (ascending)
    std::vector<double> comp_nb, comp_nc; // [ncomp] ||b_c||, ||c_c|| (weighted lower storage)
    std::vector<long long> minv_off;   // [ncomp] offset of each dense block in minv / kinv
    long long factor_size = 0;         // doubles in minv (and kinv)
    bool cached_factor = true;         // false: setup skipped the inverses (CG only)
    // cached inverses: per component a dense row-major m_c x m_c block (or, when
    // diag_factor, one value per constraint)
    std::vector<double> minv;         // (A W D^-1 A^T)^-1, Algorithms 1-2
    std::vector<double> kinv;         // (I + A W P^-1 A^T)^-1, P = I + D/2, Algorithm 3
    bool hsde_ready = false;          // kinv and the HSDE constants below are built
    // HSDE constants (Proposition 2): zeta_hat = M^-1 zeta / (1 + zeta^T M^-1 zeta);
    // its s/t parts equal +-H zhat_x / 2 and are formed on the fly.
    std::vector<double> zhat_x, zhat_y;
    double zeta_dot_zhat = 0.0;
    // The same constants for one embedding per component (each summand of a
    // direct sum embedded on its own): zeta_hat_c = M_c^-1 zeta_c / (1 + zeta_c^T M_c^-1 zeta_c)
    std::vector<double> zhat_x_c, zhat_y_c, a_zhat_x_c, zdz_c;
    std::vector<double> atb;          // A^T b per pattern entry
    std::vector<double> a_zhat_x;     // A W zhat_x per constraint
    double norm_b = 0.0, norm_c = 0.0;
    // data scaling (Section 7.1.3), when the problem was set up scaled:
    // Abar_i = e_i D A_i D, bbar = tau E b, Cbar = sigma D C D (D = diag(d))
    bool scaled = false;
    std::vector<double> sc_d, sc_e;   // [n], [m]
    double sc_tau = 1.0, sc_sigma = 1.0;
    // tau and sigma seen by each vertex and each constraint: the scalars above,
    // or, for a batch of SDPs (cdsdp_setup_batch), those of the vertex's or the
    // constraint's own SDP; sc_tau_b / sc_sigma_b per SDP (one entry otherwise)
    std::vector<double> sc_tau_v, sc_sigma_v, sc_tau_r, sc_sigma_r;
    std::vector<double> sc_tau_b, sc_sigma_b;
};

// Build everything above.  Returns a cdsdp_status.
int build_host_problem(int n, int m,
                       long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                       const double* b,
                       long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                       long long nnzP, const int* P_row, const int* P_col,
                       HostProblem& hp, bool cache_factor = true, bool merge = false);

// Cached inverse for Algorithms 1-2 (hsde = false) or 3 (hsde = true).
int build_factor(const HostProblem& hp, bool hsde, std::vector<double>& inv);

// kinv, zeta_hat and the other constants of Algorithm 3 (built on the first
// HSDE solve; primal and dual solves do not need them).
int build_hsde_constants(HostProblem& hp);

// Scaling factors of Section 7.1.3 (symmetric Ruiz equilibration of the
// constraint triplets, then b and C normalised); see cdsdp_setup_scaled.
void scaling_factors(int n, int m, long long nnzA, const int* A_con, const int* A_row, const int* A_col,
                     const double* A_val, const double* b, long long nnzC, const int* C_row, const int* C_col,
                     const double* C_val, int passes, std::vector<double>& d, std::vector<double>& e, double& tau,
                     double& sigma);

// Maximum-determinant completion (Section 7.1.1), completion.cu.  The step
// launches of the dense recurrence are replayed from a CUDA graph cached per
// (scratch, output) pair.
struct CmpGraph {
    void* exec = nullptr;  // cudaGraphExec_t
    const void* scratch = nullptr;
    const void* W = nullptr;
};
int completion_sizes(const HostProblem& hp, size_t* scratch_bytes, long long* w_elems, long long* w_offsets);
int completion_run(const HostProblem& hp, const double* d_X, void* d_scratch, size_t scratch_bytes, double* d_W,
                   double* logdet, void* stream, std::string* err, CmpGraph* cache);
void completion_release(CmpGraph& g);

inline int packed_size(int s) { return s * (s + 1) / 2; }

}  // namespace cdsdp_impl
