// Internal types shared by the host driver and the CUDA kernels of libffe.
// Nothing here is part of the public ABI (see include/ffe.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ffe.h"

namespace ffe {

constexpr int NV = 9;          // E~x E~y E~z B~x B~y B~z psi~ phi~ q~
constexpr int NG = 5;          // components of the stiff operator: E~ (3), psi~, phi~
constexpr int NJ = 6;          // stored currents: drift (3), full = drift + eta part (3)
constexpr int MAXNP = 8;       // P <= 7
constexpr int MAXNC = 15;      // 2P+1
constexpr int GH = 3;          // FD ghost layers

// Stored 3+1 metric quantities per DG node (Kerr-Schild), SoA [NMET][n_dg]:
// alpha, beta^i, gamma_ij (xx xy xz yy yz zz), gamma^ij (same), sqrt(gamma),
// d_j alpha, d_j beta^i (index 3 j + i), gamma^jk Gamma^i_jk, K.
enum MetIdx : int { M_ALPHA = 0, M_BETA = 1, M_GL = 4, M_GU = 10, M_SQRTG = 16, M_DALPHA = 17,
                    M_DBETA = 20, M_GTRACE = 29, M_K = 32, NMET = 33 };
constexpr int NPM = 17;        // the pointwise part (alpha .. sqrt(gamma)), without derivatives

// IMEX-SSP3(4,3,3) coefficients (Pareschi & Russo 2005).
constexpr double IM_A = 0.24169426078821;
constexpr double IM_B = 0.06042356519705;
constexpr double IM_H = 0.12915286960590;

// substep kinds of the device stage kernels
enum Sub : int { SUB_A = 0, SUB_B = 1, SUB_C = 2, SUB_RHS = 3 };

// 1-D operator tables of one order P (built on the host in long double).
struct Tables {
    int P, np1, nc;
    double x[MAXNP], w[MAXNP], w0;
    double D[MAXNP][MAXNP];        // D_ij = l_j'(x_i)
    double Filt[MAXNP][MAXNP];     // V diag(sigma) V^-1
    // Filt = I - sum_r FrV[r] FrW[r]^T over the nfr modes m the filter damps by
    // more than 1e-20 (FrV[r][i] = P_m(x_i), FrW[r][j] = (1 - sigma_m) (V^-1)[m][j])
    int nfr;
    double FrV[MAXNP][MAXNP], FrW[MAXNP][MAXNP];
    double Pi[MAXNP][MAXNP];       // projection on Legendre modes p <= P - M
    double P2F[MAXNC][MAXNP];      // DG -> FD (Lagrange evaluation at subcell centres)
    double F2D[MAXNP][MAXNC];      // FD -> DG (6-point Lagrange, shifted inside)
    int f2d_lo[MAXNP];             // first subcell of the 6-point stencil of node i
};

// Per-instance data of a batched context (one magnetosphere per instance).
struct InstInfo {
    double r_in, c, dt, omega;   // shell map r = r_in exp(c (er + 1)), time step, star rotation
    int na, nr, e0, P;           // elements per wedge side / radially, first element, order
    int tab;                     // offset of the instance's FD-point tables in Dev::stab
};

// A field buffer in state-vector layout: [nv][n_dg] then [nv][n_fd].
struct Field {
    double* p;
    int nv;
    int64_t ndg, nfd;
    __host__ __device__ double* dg(int v) const { return p + (int64_t)v * ndg; }
    __host__ __device__ double* fd(int v) const { return p + (int64_t)nv * ndg + (int64_t)v * nfd; }
};

// Everything a kernel needs to know about the context (passed by value).
struct Dev {
    // E elements; P, np1, nc are the largest order's sizes and nn, ncell the
    // node / cell slot of every element (elements of lower order use the front
    // of their slot); uniform contexts have one order.
    int E, P, np1, nn, nc, ncell;
    int64_t ndg, nfd;
    int nsm;                        // streaming multiprocessors of the device (launch shapes)
    const unsigned char* eP;        // [E] order of each element (null: all P)
    const int* einst;               // [E] instance of each element (null: one instance)
    const InstInfo* inst;           // [n_inst]
    const Tables* tabs;             // [MAXNP] tables indexed by order
    double thr_dgP[MAXNP], thr_fdP[MAXNP];   // indicator thresholds per order
    // FD storage: slot of each element ([E], -1 if none) and element of each
    // slot; null = slot e for element e.  Free slots form a stack.
    int* fd_slot;
    int* slot_elem;
    int* free_slots;
    int fd_cap;                     // FD slots
    int chunk;                      // FD elements per scratch chunk
    int dg_grid;                    // CTAs of the DG kernel of the highest order (autotuner; 0 = default)
    int dg_grid_lo, dg_grid_lo2;    // batches: CTAs of the DG kernels of orders P-1, P-2 (autotuner; 0 = default)
    // physics and scheme parameters
    double eta, kpsi, kphi, dt, weno_eps, omega;
    int mode, filter_on, tci_on, fd_corr, recon;
    double thr_dg, thr_fd;          // (P+1-M)^-alpha and (P+1-M)^-(alpha+1)
    // geometry of the affine box: d xi / d x per element and axis
    const double* ijac;             // [E][3]
    // curved meshes: d xi^k / d x^i per DG node [9][ndg] (index 3 k + i), the
    // Kerr-Schild metric per DG node [NMET][ndg] (null in flat space), and the
    // shell map for FD cells and faces (closed form, from stab)
    int curved, ks;
    const double* geo;
    const double* met;
    // Kerr-Schild metric at FD points (null in flat space): subcell centres
    // [NMET][E ncell]; face points [3][NPM][E (nc+1) nc^2]; ghost centres across
    // Dirichlet faces [nbf][NPM][GH nc^2]
    const double* metfd;
    const double* metff;
    const double* metgb;
    // faces between cubed-sphere wedges: ghost-table slot of each element face
    // ([E][6], -1 elsewhere) and per ghost (slot, g, ta, tb) of the slot's face,
    // [slot][GH nc^2]: the first neighbour cell of its 6-point stencil along each
    // axis [3] with the stencil weights [3][6], and the Lagrange weights of the
    // neighbour's LGL nodes along each axis [3][MAXNP]
    const int* gislot;
    const int* gst;
    const double* gwf;
    const double* gwl;
    const int* gbox;                // [slot][6]: first neighbour cell and extent of the stencils' box per axis
    int gbox_max;                   // largest box volume (cells)
    double shell_rin, shell_c;
    int shell_na, shell_nr;
    // flat shells, per instance at InstInfo::tab (single context: 0), on the
    // half-cell grid g = 2 nc i + h of each angular / radial element row (h even:
    // FD faces, h odd: cell centres): X_g = tan(pi/4 e_g), 1/(pi/4 (1 + X_g^2))
    // [2 nc na + 1 each], then r_g, 1/r_g [2 nc nr + 1 each]
    const double* stab;
    const double* xyz_dg;           // [3][ndg] node coordinates
    const double* xyz_fd;           // [3][xfd_n] subcell-centre coordinates of every element
                                    // (element e's cells at e ncell; null in batches)
    int64_t xfd_n;
    // connectivity
    const int* nbr;                 // [E][6] neighbour element or -1
    const int* nbr_face;            // [E][6] the neighbour's face touching mine
    const int* orient;              // [E][6] orientation code of the shared face (shellmap.cuh)
    const int* bc;                  // [E][6] boundary kind when nbr < 0
    const unsigned char* ginterp;   // [E][6] 1: face between cubed-sphere wedges, FD ghosts
                                    // interpolated to the extended grid (null: none)
    const int* bface;               // [E][6] boundary-face slot (Dirichlet data) or -1
    const double* bdg;              // [nbf][9][np1*np1] Dirichlet states at face nodes
    const double* bfd;              // [nbf][9][GH][nc*nc] Dirichlet states in ghost cells
    const Tables* tab;              // tables of order P
    // mask, lists and counters (device)
    unsigned char* mask;            // [E] 0 = DG, 1 = FD
    unsigned char* switched;        // [E] switched to FD during the current step
    int* dg_list; int* fd_list; int* flag_list; int* near_list;
    int* dg_list_lo;   // batches: DG elements of order P-1 (count in counts[6]); null otherwise
    int* dg_list_lo2;  // batches: DG elements of order P-2 (count in counts[7]); null otherwise
    int* counts;                    // [0] n_dg, [1] n_fd, [2] n_flag, [3] n_near, [4] status bits, [5] free slots
    unsigned long long* units;      // [0] node updates (DG nodes + FD cells per substep), [1] FD and [2] DG element updates
    // FD scratch per chunk of listed FD elements: extended cells [12][chunk][(nc+6)^3],
    // face fluxes [3 (x3 curved)][9][chunk][(nc+1) nc^2]
    double* ext;
    double* flux;
    // FD->DG face traces of FD elements for their DG neighbours, per FD slot
    // [6][12][np1^2] (k_fd_traces; null: none), and their adjoints in the
    // reverse mode (written by the DG reverse kernel, allocated with the adjoint)
    double* ftr;
    double* ftr_b;
};

// sizes of one element
struct ES {
    int P, np1, nn, nc, ncell;
};
__host__ __device__ inline ES es_of(int P) {
    ES s;
    s.P = P;
    s.np1 = P + 1;
    s.nn = s.np1 * s.np1 * s.np1;
    s.nc = 2 * P + 1;
    s.ncell = s.nc * s.nc * s.nc;
    return s;
}
__device__ __forceinline__ int elem_P(const Dev& d, int e) { return d.eP ? (int)d.eP[e] : d.P; }
__device__ __forceinline__ ES esz(const Dev& d, int e) { return es_of(elem_P(d, e)); }
__device__ __forceinline__ int64_t fdb(const Dev& d, int e) {
    return (int64_t)(d.fd_slot ? d.fd_slot[e] : e) * d.ncell;
}
__device__ __forceinline__ int fd_slot_of(const Dev& d, int e) { return d.fd_slot ? d.fd_slot[e] : e; }
__device__ __forceinline__ double dt_of(const Dev& d, int e) { return d.einst ? d.inst[d.einst[e]].dt : d.dt; }
__device__ __forceinline__ double omega_of(const Dev& d, int e) { return d.einst ? d.inst[d.einst[e]].omega : d.omega; }

// kernel launchers (kernels_*.cu); all enqueue on `st`
void launch_build_lists(const Dev& d, cudaStream_t st);
void launch_current(const Dev& d, Field U, Field J, const int* list_or_null, int which_count, cudaStream_t st);
void launch_stage12(const Dev& d, Field un, Field Ua, Field G1, Field G2, cudaStream_t st);
void launch_dg_substep(const Dev& d, int sub, Field Uin, Field J, Field un, Field F2, Field F3,
                       Field G1, Field G2, Field G3, Field G4, Field Fout, Field Uout, Field Gout,
                       cudaStream_t st);
void launch_fd_substep(const Dev& d, int sub, const int* list, int count_index, Field Uin, Field J,
                       Field un, Field F2, Field F3, Field G1, Field G2, Field G3, Field G4,
                       Field Fout, Field Uout, Field Gout, cudaStream_t st);
int fd_chunks(const Dev& d);
// FD->DG face traces of the listed FD elements for their DG neighbours (Dev::ftr)
void launch_fd_traces(const Dev& d, Field U, Field J, cudaStream_t st);
// out += the FD cells' share of the trace adjoints (Dev::ftr_b), reverse of k_fd_traces
void launch_fd_traces_vjp(const Dev& d, Field U, Field out, cudaStream_t st);
// extended blocks (U, J~ with ghosts) of the listed FD elements of one chunk
void launch_fd_fill(const Dev& d, const int* list, int count_index, int w0, Field U, Field J, cudaStream_t st);
void launch_eval_recip(const double* x, double* y, int64_t n, cudaStream_t st);
// register-only DFMA loop: returns its flops, *ms its event-timed duration
double launch_fma_probe(int nsm, int iters, cudaStream_t st, float* ms);
// ghosts of the faces between cubed-sphere wedges (kernels_fd_interp.cu)
void launch_fd_fill_interp(const Dev& d, const int* list, int ci, int w0, Field U, Field J, cudaStream_t st);
void launch_fdv_ghosts_interp(const Dev& d, const int* list, int ci, int w0, Field U, Field out, const double* extb,
                              cudaStream_t st);
void launch_constraints(const Dev& d, Field U, double* part, int blocks, cudaStream_t st);
void launch_l2_err(const Dev& d, Field U, Field R, int v0, int nv, double* part, int blocks, cudaStream_t st);
// out += (d RHS_FD/dU)^T L (kernels_adjoint_fd.cu); extb: scratch of the size of d.ext
// FD elements per chunk of the FD reverse mode (its per-face buffer gb holds
// [3][12][FDV_CHUNK][(nc+1) nc^2][6] doubles)
constexpr int FDV_CHUNK = 1024;
void launch_fd_rhs_vjp(const Dev& d, Field U, Field J, Field L, Field out, double* extb, double* gb,
                       double* omega_bar, cudaStream_t st);
void launch_rollback_project(const Dev& d, int sub, Field un, Field Uin, Field F2, Field F3,
                             Field G1, Field G2, Field G3, Field G4, cudaStream_t st);
void launch_fd2dg(const Dev& d, Field un, cudaStream_t st);
void launch_tci_ratio(const Dev& d, const double* Udg, double* ratio, cudaStream_t st);
void launch_dg_substep_curved(const Dev& d, int sub, Field Uin, Field J, Field un, Field F2, Field F3, Field G1,
                              Field G2, Field G3, Field G4, Field Fout, Field Uout, Field Gout, cudaStream_t st);
void launch_stage12_ks(const Dev& d, Field un, Field Ua, Field G1, Field G2, cudaStream_t st);

// adjoint (kernels_adjoint.cu)
struct AdjArgs {
    Field un, U2, R3, R4, T3, T4, U3, U4, F2, F3, F4, G1, G2, G3, G4, W;
    Field lam, ubar, F2b, F3b, F4b, G1b, G2b, G3b, G4b, tmp, tmp2;
};
void launch_rhs_vjp(const Dev& d, Field U, Field L, Field out, double* omega_bar, cudaStream_t st);
void launch_filter(const Dev& d, Field in, Field out, int nv, int transpose, cudaStream_t st);
void launch_adj(const Dev& d, int which, AdjArgs a, int sub, cudaStream_t st);
void launch_adj_addG(const Dev& d, Field U, Field Gb, Field io, cudaStream_t st);
void launch_adj_clamp(const Dev& d, Field io, cudaStream_t st);
void launch_adj_clamp_back(const Dev& d, Field X, Field yb, Field out, cudaStream_t st);
void launch_luminosity(const Dev& d, Field U, const int* elem, const double* lk, const double* wn, int ns,
                       double* partial, int nblocks, Field grad, double scale, cudaStream_t st, int bflux = 0);

extern thread_local int64_t g_launch_counter;

// optional per-kernel event timing (host.cu); no-ops unless profiling is on
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);

}  // namespace ffe
