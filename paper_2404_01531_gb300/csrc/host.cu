// Host side of libffe: operator tables, mesh and geometry, initial data,
// context lifetime, the IMEX step driver (captured once into a CUDA graph) and
// the C ABI declared in include/ffe.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <map>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include "ffe_internal.h"
#include "geom_host.h"
#include "shellmap.cuh"

using namespace ffe;

namespace {

thread_local std::string g_err;

ffe_status fail(ffe_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

// Every entry point's body is a function-try-block ending here, so that no C++
// exception (a failed host allocation, a host thread that cannot be started)
// crosses the C ABI: it becomes FFE_ENOMEM with its description.  A context
// being created when that happens is not released.
ffe_status host_failure() {
    try {
        throw;
    } catch (const std::exception& ex) {
        return fail(FFE_ENOMEM, "host resources exhausted: %s", ex.what());
    } catch (...) {
        return fail(FFE_ENOMEM, "host resources exhausted");
    }
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t _e = (call);                                                          \
        if (_e != cudaSuccess)                                                            \
            return fail(FFE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(_e));       \
    } while (0)

// ---------------------------------------------------------------- tables ----
typedef long double ld;

void legendre(int n, ld x, ld& L, ld& dL) {
    ld p0 = 1.0L, p1 = x;
    if (n == 0) { L = 1.0L; dL = 0.0L; return; }
    for (int k = 1; k < n; ++k) {
        ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    L = p1;
    if (fabsl(x) == 1.0L) dL = (x > 0 ? 1.0L : ((n + 1) % 2 ? -1.0L : 1.0L)) * n * (n + 1) / 2.0L;
    else dL = n * (p0 - x * p1) / (1.0L - x * x);
}

// LGL points: +-1 and the zeros of L_N', by Newton from Chebyshev-Lobatto guesses.
void lgl(int N, std::vector<ld>& x, std::vector<ld>& w) {
    x.assign(N + 1, 0.0L);
    w.assign(N + 1, 0.0L);
    x[0] = -1.0L;
    x[N] = 1.0L;
    for (int j = 1; j < N; ++j) {
        ld t = -cosl(3.14159265358979323846264338327950288L * j / N);
        for (int it = 0; it < 100; ++it) {
            ld L, dL;
            legendre(N, t, L, dL);
            ld d2 = (2 * t * dL - N * (N + 1) * L) / (1 - t * t);
            ld dt = dL / d2;
            t -= dt;
            if (fabsl(dt) < 1e-19L) break;
        }
        x[j] = t;
    }
    for (int j = 0; j <= N / 2; ++j) {   // symmetrise
        ld m = 0.5L * (x[N - j] - x[j]);
        x[j] = -m;
        x[N - j] = m;
    }
    for (int j = 0; j <= N; ++j) {
        ld L, dL;
        legendre(N, x[j], L, dL);
        w[j] = 2.0L / (N * (N + 1) * L * L);
    }
}

bool invert(std::vector<ld>& A, int n) {   // Gauss-Jordan with partial pivoting, in place
    std::vector<ld> I(n * n, 0.0L);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0L;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0L) return false;
        for (int k = 0; k < n; ++k) { std::swap(A[c * n + k], A[p * n + k]); std::swap(I[c * n + k], I[p * n + k]); }
        ld piv = A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] /= piv; I[c * n + k] /= piv; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ld f = A[r * n + c];
            for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
        }
    }
    A = I;
    return true;
}

ld lagrange(const std::vector<ld>& xs, int j, ld y) {
    ld r = 1.0L;
    for (size_t m = 0; m < xs.size(); ++m)
        if ((int)m != j) r *= (y - xs[m]) / (xs[j] - xs[m]);
    return r;
}

void build_tables(int P, double fa, double fb, int M, Tables& T) {
    memset(&T, 0, sizeof T);
    const int np1 = P + 1, nc = 2 * P + 1;
    T.P = P;
    T.np1 = np1;
    T.nc = nc;
    std::vector<ld> x, w;
    lgl(P, x, w);
    for (int i = 0; i < np1; ++i) { T.x[i] = (double)x[i]; T.w[i] = (double)w[i]; }
    T.w0 = (double)w[0];
    std::vector<ld> L(np1);
    for (int i = 0; i < np1; ++i) { ld dl; legendre(P, x[i], L[i], dl); }
    for (int i = 0; i < np1; ++i)
        for (int j = 0; j < np1; ++j)
            T.D[i][j] = (i != j) ? (double)(L[i] / (L[j] * (x[i] - x[j]))) : 0.0;
    T.D[0][0] = -P * (P + 1) / 4.0;
    T.D[P][P] = P * (P + 1) / 4.0;
    std::vector<ld> V(np1 * np1), Vi;
    for (int i = 0; i < np1; ++i)
        for (int j = 0; j < np1; ++j) { ld l, dl; legendre(j, x[i], l, dl); V[i * np1 + j] = l; }
    Vi = V;
    invert(Vi, np1);
    for (int i = 0; i < np1; ++i)
        for (int j = 0; j < np1; ++j) {
            ld sf = 0.0L, sp = 0.0L;
            for (int m = 0; m < np1; ++m) {
                ld sig = expl(-(ld)fa * powl((ld)m / P, 2.0L * (ld)fb));
                ld keep = (m <= P - M) ? 1.0L : 0.0L;
                sf += V[i * np1 + m] * sig * Vi[m * np1 + j];
                sp += V[i * np1 + m] * keep * Vi[m * np1 + j];
            }
            T.Filt[i][j] = (double)sf;
            T.Pi[i][j] = (double)sp;
        }
    // low-rank form of the filter: modes damped by 1 - sigma_m > 1e-20 (the rest
    // change a nodal value by less than 1e-20 of the mode's coefficient)
    std::vector<int> damped;
    for (int m = 0; m < np1; ++m)
        if (-expm1l(-(ld)fa * powl((ld)m / P, 2.0L * (ld)fb)) > 1e-20L) damped.push_back(m);
    T.nfr = (int)damped.size();
    for (int r = 0; r < T.nfr; ++r) {
        const int m = damped[r];
        const ld dm = -expm1l(-(ld)fa * powl((ld)m / P, 2.0L * (ld)fb));
        for (int i = 0; i < np1; ++i) {
            T.FrV[r][i] = (double)V[i * np1 + m];
            T.FrW[r][i] = (double)(dm * Vi[m * np1 + i]);
        }
    }
    std::vector<ld> xc(nc);
    const ld dxi = 2.0L / nc;
    for (int c = 0; c < nc; ++c) xc[c] = -1.0L + (c + 0.5L) * dxi;
    for (int c = 0; c < nc; ++c)
        for (int j = 0; j < np1; ++j) T.P2F[c][j] = (double)lagrange(x, j, xc[c]);
    if (nc >= 6) {
        for (int i = 0; i < np1; ++i) {
            ld pos = (x[i] + 1.0L) / dxi - 0.5L;
            int lo = (int)floorl(pos) - 2;
            lo = lo < 0 ? 0 : (lo > nc - 6 ? nc - 6 : lo);
            T.f2d_lo[i] = lo;
            std::vector<ld> st(xc.begin() + lo, xc.begin() + lo + 6);
            for (int m = 0; m < 6; ++m) T.F2D[i][lo + m] = (double)lagrange(st, m, x[i]);
        }
    }
}

// ------------------------------------------------------------ initial data --
void initial_point(int kind, const double* prm, int nprm, const double* X, double* U) {
    for (int v = 0; v < NV; ++v) U[v] = 0.0;
    const double x = X[0];
    if (kind == FFE_ID_FAST_WAVE) {
        double amp = nprm > 0 ? prm[0] : 0.5;
        double b = 1.0 + amp * sin(M_PI * x);
        U[3] = 1.0;
        U[4] = b;
        U[2] = -b;
    } else if (kind == FFE_ID_BREAKDOWN) {
        U[3] = 1.0;
        U[4] = x < -0.1 ? 1.0 : (x > 0.1 ? -1.0 : -10.0 * x);
        U[2] = fabs(x) < 0.1 ? 0.5 : 1.0;
    } else if (kind == FFE_ID_CLEANING_MODE) {
        double eps = nprm > 0 ? prm[0] : 1e-3;
        U[3] = 1.0 + eps * sin(M_PI * x);
    } else if (kind == FFE_ID_WALD) {
        wald_point(X, nprm > 0 ? prm[0] : 1.0, nprm > 1 ? prm[1] : 0.0, nprm > 2 ? prm[2] : 1.0, U);
        // optional fourth parameter: a factor on E~ (0: the vacuum Wald problem's
        // start, Wald's B~ with E~ = 0, Sec. IV.B.2)
        if (nprm > 3)
            for (int v = 0; v < 3; ++v) U[v] *= prm[3];
    } else if (kind == FFE_ID_DIPOLE) {
        dipole_point(X, nprm > 0 ? prm[0] : 1.0, nprm > 1 ? prm[1] : 0.1, nprm > 2 ? prm[2] : 0.0, U);
    } else if (kind == FFE_ID_FAST_WAVE_KINK) {
        // App. A fast wave: B = (1, b, 0), E = (0, 0, -b), b = 1 | 0.85 - 1.5 x | 0.7
        const double b = x < -0.1 ? 1.0 : (x > 0.1 ? 0.7 : 0.85 - 1.5 * x);
        U[3] = 1.0;
        U[4] = b;
        U[2] = -b;
    } else if (kind == FFE_ID_ALFVEN) {
        // App. A stationary Alfven wave: B = (1, 1, b), E = (-b, 0, 1),
        // b = 1 | 1.15 + 0.15 sin(5 pi x) | 1.3; q~ = div E~ = -db/dx
        const bool in = fabs(x) < 0.1;
        const double b = x < -0.1 ? 1.0 : (x > 0.1 ? 1.3 : 1.15 + 0.15 * sin(5.0 * M_PI * x));
        U[0] = -b;
        U[2] = 1.0;
        U[3] = 1.0;
        U[4] = 1.0;
        U[5] = b;
        U[8] = in ? -0.75 * M_PI * cos(5.0 * M_PI * x) : 0.0;
    } else if (kind == FFE_ID_BREAKDOWN_1D) {
        // App. A FFE breakdown: B = (1, b, b), E = (0, 0.5, -0.5), b = 1 | -10 x | -1
        const double b = x < -0.1 ? 1.0 : (x > 0.1 ? -1.0 : -10.0 * x);
        U[1] = 0.5;
        U[2] = -0.5;
        U[3] = 1.0;
        U[4] = b;
        U[5] = b;
    }
}

// run fn(i) for i in [0, n) on all host cores; a share whose thread cannot be
// started runs on the calling thread (the started ones are always joined)
template <typename F>
void parallel_for(int64_t n, F fn) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt == 0 ? 1 : (nt > 64 ? 64 : nt);
    std::vector<std::thread> th;
    th.reserve(nt);
    for (unsigned t = 0; t < nt; ++t) {
        auto share = [&, t]() {
            for (int64_t i = t; i < n; i += nt) fn(i);
        };
        try {
            th.emplace_back(share);
        } catch (...) {
            share();
        }
    }
    for (auto& x : th) x.join();
}

// ---------------------------------------------------------------- profiler --
struct ProfRec { std::string name; cudaEvent_t a, b; };
struct Profiler {
    bool on = false;
    std::vector<ProfRec> pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
    size_t used = 0;
    struct Tot { long n; double ms, max_ms; };
    std::vector<std::pair<std::string, Tot>> totals;
    void add(const std::string& n, double ms) {
        for (auto& t : totals)
            if (t.first == n) {
                t.second.n += 1;
                t.second.ms += ms;
                t.second.max_ms = ms > t.second.max_ms ? ms : t.second.max_ms;
                return;
            }
        totals.push_back({n, {1, ms, ms}});
    }
};
thread_local Profiler g_prof;

}  // namespace

namespace ffe {
void prof_begin(const char* name, cudaStream_t st) {
    if (!g_prof.on) return;
    if (g_prof.used == g_prof.pool.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        g_prof.pool.push_back({a, b});
    }
    auto& ev = g_prof.pool[g_prof.used++];
    g_prof.pending.push_back({name, ev.first, ev.second});
    cudaEventRecord(ev.first, st);
}
void prof_end(cudaStream_t st) {
    if (!g_prof.on || g_prof.pending.empty()) return;
    cudaEventRecord(g_prof.pending.back().b, st);
}
}  // namespace ffe

namespace {
void prof_collect(cudaStream_t st) {
    if (!g_prof.on) return;
    cudaStreamSynchronize(st);
    for (auto& r : g_prof.pending) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        g_prof.add(r.name, ms);
    }
    g_prof.pending.clear();
    g_prof.used = 0;
}
}  // namespace

// ------------------------------------------------------------- context ------
struct ffe_ctx {
    ffe_domain dom;
    ffe_elements el;
    ffe_metric met;
    ffe_params prm;
    cudaStream_t st = nullptr;
    Dev d{};
    Tables tab{};
    int nx = 0, ny = 0, nz = 0;
    double h[3] = {0, 0, 0};
    double dxmin = 0.0, t = 0.0;
    int64_t steps = 0;
    int id_kind = -1;
    std::vector<double> id_prm;
    std::vector<void*> allocs;
    Field un{}, Ua{}, Ub{}, F2{}, F3{}, G1{}, G2{}, G3{}, G4{}, J{}, Fs{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = true;
    int graph_kernels = 0;
    int nbf = 0;                     // boundary faces with Dirichlet data
    std::vector<int> h_bface;
    std::vector<unsigned char> h_ginterp;   // [E][6] faces between cubed-sphere wedges
    std::vector<int> h_gislot;              // [E][6] their ghost-table slot (-1 elsewhere)
    ShellGeo shell{};
    double lam_max = 1.0;
    // batched contexts
    bool batch = false;
    int n_inst = 1;
    std::vector<InstInfo> insts;          // per instance
    std::vector<ffe_domain> doms;
    std::vector<int> h_eP, h_einst;       // per element
    std::vector<int> h_fd_slot;           // per element (pool only)
    std::vector<double> id_prm_inst;      // initial-data parameters per instance
    int id_nprm = 0;
    Tables tabs_h[MAXNP];
    bool tuned = false;
    // adjoint work fields (allocated by the first adjoint call)
    bool adj_ready = false;
    int tci_param = 0;               // the indicator setting of ffe_create
    AdjArgs adj{};
    bool adj_fd = false;             // the current mask has FD elements
    double* d_extb = nullptr;        // extended-block adjoint of one FD chunk
    double* d_gbuf = nullptr;        // per-face contributions to it (FD reverse mode)
    double* d_omega_bar = nullptr;
    double* d_cons = nullptr;        // per-block partials of ffe_constraints
    double* d_ref = nullptr;         // analytic initial data (reference of the L2 error), state layout
    bool ref_valid = false;          // d_ref matches the current mask, FD slots and initial data
    std::vector<unsigned char> ref_mask;
    std::vector<int> ref_slot;
    double* d_partial = nullptr;
    // surface quadratures of the luminosity and the upper-half magnetic flux,
    // cached per (radius, upper half only, instance of a batch or -1)
    struct Surf {
        int ns = 0;
        int* elem = nullptr;
        double* lk = nullptr;
        double* w = nullptr;
    };
    std::map<std::tuple<double, int, int>, Surf> surf;
};

namespace {

template <typename T>
ffe_status dalloc(ffe_ctx* c, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 1);
    if (e != cudaSuccess) return fail(FFE_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    cudaMemset(q, 0, n * sizeof(T));
    c->allocs.push_back(q);
    *p = (T*)q;
    return FFE_OK;
}

ffe_status alloc_field(ffe_ctx* c, Field& f, int nv) {
    f.nv = nv;
    f.ndg = c->d.ndg;
    f.nfd = c->d.nfd;
    return dalloc(c, &f.p, (size_t)nv * (f.ndg + f.nfd));
}

int elem_id(const ffe_ctx* c, int ex, int ey, int ez) { return ex + c->nx * (ey + c->ny * ez); }

// Build the affine box mesh, connectivity and coordinates on the host and upload.
ffe_status build_box(ffe_ctx* c) {
    const int E = c->d.E, np1 = c->d.np1, nc = c->d.nc, nn = c->d.nn, ncell = c->d.ncell;
    const int n[3] = {c->nx, c->ny, c->nz};
    std::vector<double> ijac(3 * E), xdg(3 * (size_t)c->d.ndg), xfd(3 * (size_t)c->d.nfd);
    std::vector<int> nbr(6 * E, -1), nbf(6 * E, -1), bc(6 * E, 0), bface(6 * E, -1);
    int nbfd = 0;
    for (int ez = 0; ez < c->nz; ++ez)
        for (int ey = 0; ey < c->ny; ++ey)
            for (int ex = 0; ex < c->nx; ++ex) {
                const int e = elem_id(c, ex, ey, ez);
                const int ix[3] = {ex, ey, ez};
                for (int dd = 0; dd < 3; ++dd) ijac[3 * e + dd] = 2.0 / c->h[dd];
                for (int f = 0; f < 6; ++f) {
                    const int dd = f >> 1, s = f & 1;
                    int jx[3] = {ix[0], ix[1], ix[2]};
                    jx[dd] += s ? 1 : -1;
                    const int kind = s ? c->dom.bc_hi[dd] : c->dom.bc_lo[dd];
                    if (jx[dd] < 0 || jx[dd] >= n[dd]) {
                        if (kind == FFE_BC_PERIODIC) jx[dd] = (jx[dd] + n[dd]) % n[dd];
                        else {
                            bc[6 * e + f] = kind;
                            if (kind == FFE_BC_DIRICHLET) bface[6 * e + f] = nbfd++;
                            continue;
                        }
                    }
                    nbr[6 * e + f] = elem_id(c, jx[0], jx[1], jx[2]);
                    nbf[6 * e + f] = 2 * dd + (1 - s);
                }
                for (int k = 0; k < np1; ++k)
                    for (int j = 0; j < np1; ++j)
                        for (int i = 0; i < np1; ++i) {
                            const int64_t p = (int64_t)e * nn + i + np1 * (j + np1 * k);
                            const double xi[3] = {c->tab.x[i], c->tab.x[j], c->tab.x[k]};
                            for (int dd = 0; dd < 3; ++dd)
                                xdg[dd * c->d.ndg + p] = c->dom.lo[dd] + (ix[dd] + 0.5 * (xi[dd] + 1.0)) * c->h[dd];
                        }
                for (int z = 0; z < nc; ++z)
                    for (int y = 0; y < nc; ++y)
                        for (int x = 0; x < nc; ++x) {
                            const int64_t p = (int64_t)e * ncell + x + nc * (y + nc * z);
                            const int cc[3] = {x, y, z};
                            for (int dd = 0; dd < 3; ++dd) {
                                const double xi = -1.0 + (cc[dd] + 0.5) * 2.0 / nc;
                                xfd[dd * c->d.nfd + p] = c->dom.lo[dd] + (ix[dd] + 0.5 * (xi + 1.0)) * c->h[dd];
                            }
                        }
            }
    c->nbf = nbfd;
    c->h_bface = bface;
    double *d_ijac, *d_xdg, *d_xfd, *d_bdg, *d_bfd;
    int *d_nbr, *d_nbf, *d_bc, *d_bface;
    ffe_status s;
    if ((s = dalloc(c, &d_ijac, ijac.size()))) return s;
    if ((s = dalloc(c, &d_xdg, xdg.size()))) return s;
    if ((s = dalloc(c, &d_xfd, xfd.size()))) return s;
    if ((s = dalloc(c, &d_nbr, nbr.size()))) return s;
    if ((s = dalloc(c, &d_nbf, nbf.size()))) return s;
    if ((s = dalloc(c, &d_bc, bc.size()))) return s;
    if ((s = dalloc(c, &d_bface, bface.size()))) return s;
    if ((s = dalloc(c, &d_bdg, (size_t)(nbfd > 0 ? nbfd : 1) * NV * np1 * np1))) return s;
    if ((s = dalloc(c, &d_bfd, (size_t)(nbfd > 0 ? nbfd : 1) * NV * GH * nc * nc))) return s;
    CK(cudaMemcpy(d_ijac, ijac.data(), ijac.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_xdg, xdg.data(), xdg.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_xfd, xfd.data(), xfd.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_nbf, nbf.data(), nbf.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_bc, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_bface, bface.data(), bface.size() * 4, cudaMemcpyHostToDevice));
    int* d_or;
    if ((s = dalloc(c, &d_or, 6 * (size_t)E))) return s;
    c->d.orient = d_or;
    c->d.ijac = d_ijac;
    c->d.xyz_dg = d_xdg;
    c->d.xyz_fd = d_xfd;
    c->d.xfd_n = (int64_t)c->d.E * c->d.ncell;
    c->d.nbr = d_nbr;
    c->d.nbr_face = d_nbf;
    c->d.bc = d_bc;
    c->d.bface = d_bface;
    c->d.bdg = d_bdg;
    c->d.bfd = d_bfd;
    // (dx)_min: smallest gap between adjacent LGL nodes along any element line
    double gap = 1e300;
    for (int i = 0; i < np1 - 1; ++i) gap = fmin(gap, c->tab.x[i + 1] - c->tab.x[i]);
    c->dxmin = 1e300;
    for (int dd = 0; dd < 3; ++dd) c->dxmin = fmin(c->dxmin, 0.5 * c->h[dd] * gap);
    return FFE_OK;
}

// x(xi) and d xi / d x of element e for either mesh kind.
MapFn ctx_map(ffe_ctx* c) {
    if (c->batch) {
        std::vector<InstInfo> in = c->insts;
        std::vector<int> ei = c->h_einst;
        return [in, ei](int e, const double xi[3], double x[3], double ij[3][3]) {
            const InstInfo& q = in[ei[e]];
            ShellGeo g{q.r_in, q.c, q.na, q.nr};
            shell_map(g, e - q.e0, xi, x, ij);
        };
    }
    if (c->dom.kind == FFE_DOMAIN_SHELL6) {
        ShellGeo g = c->shell;
        return [g](int e, const double xi[3], double x[3], double ij[3][3]) { shell_map(g, e, xi, x, ij); };
    }
    const int nx = c->nx, ny = c->ny;
    const double lo[3] = {c->dom.lo[0], c->dom.lo[1], c->dom.lo[2]}, h[3] = {c->h[0], c->h[1], c->h[2]};
    return [=](int e, const double xi[3], double x[3], double ij[3][3]) {
        const int ix[3] = {e % nx, (e / nx) % ny, e / (nx * ny)};
        for (int q = 0; q < 3; ++q) {
            x[q] = lo[q] + (ix[q] + 0.5 * (xi[q] + 1.0)) * h[q];
            for (int r = 0; r < 3; ++r) ij[q][r] = q == r ? 2.0 / h[q] : 0.0;
        }
    };
}

int host_P(const ffe_ctx* c, int e) { return c->batch ? c->h_eP[e] : c->d.P; }

// Kerr-Schild metric at the FD points of every element (the FD kernels read
// it there as the DG kernels read it at their nodes): subcell centres with the
// derivative terms of the sources, [NMET][E ncell] (Dev::metfd); face points
// of the three directions, [3][NPM][E nface] (Dev::metff; face m between cells
// m-1 and m, tangential cell centres ta, tb along axes_of); ghost centres
// across Dirichlet faces, [nbf][NPM][GH nc^2] (Dev::metgb, indexed like the
// Dirichlet ghost states).  Ghosts across faces between wedges need no metric:
// they take the neighbour's transferred current.  NPM: alpha, beta^i,
// gamma_ij, gamma^ij, sqrt(gamma), the first NPM entries of NMET.
ffe_status build_ks_fd_tables(ffe_ctx* c, const std::vector<double>& xfd) {
    Dev& d = c->d;
    const int E = d.E, nc = d.nc, ncell = d.ncell;
    const int64_t nfc = (int64_t)(nc + 1) * nc * nc, ncells = (int64_t)E * ncell, nfaces = (int64_t)E * nfc;
    const double M = c->met.M, a = c->met.a, dxi = 2.0 / nc;
    MapFn map = ctx_map(c);
    ffe_status s;
    std::vector<double> mc((size_t)NMET * ncells);
    parallel_for(ncells, [&](int64_t p) {
        double x[3] = {xfd[p], xfd[ncells + p], xfd[2 * ncells + p]}, out[NMET];
        ks_point(x, M, a, out);
        for (int q = 0; q < NMET; ++q) mc[q * ncells + p] = out[q];
    });
    double* d_mc;
    if ((s = dalloc(c, &d_mc, mc.size()))) return s;
    CK(cudaMemcpy(d_mc, mc.data(), mc.size() * 8, cudaMemcpyHostToDevice));
    std::vector<double>().swap(mc);
    d.metfd = d_mc;
    std::vector<double> mf((size_t)3 * NPM * nfaces);
    parallel_for(E, [&](int64_t e) {
        for (int k = 0; k < 3; ++k) {
            const int t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
            for (int64_t fi = 0; fi < nfc; ++fi) {
                const int m = (int)(fi % (nc + 1)), ta = (int)((fi / (nc + 1)) % nc), tb = (int)(fi / ((nc + 1) * nc));
                double xi[3], x[3], ij[3][3], out[NMET];
                xi[k] = -1.0 + m * dxi;
                xi[t1] = -1.0 + (ta + 0.5) * dxi;
                xi[t2] = -1.0 + (tb + 0.5) * dxi;
                map((int)e, xi, x, ij);
                ks_point(x, M, a, out);
                for (int q = 0; q < NPM; ++q) mf[((size_t)k * NPM + q) * nfaces + e * nfc + fi] = out[q];
            }
        }
    });
    double* d_mf;
    if ((s = dalloc(c, &d_mf, mf.size()))) return s;
    CK(cudaMemcpy(d_mf, mf.data(), mf.size() * 8, cudaMemcpyHostToDevice));
    std::vector<double>().swap(mf);
    d.metff = d_mf;
    // ghost centres: the element's reference grid continued past the face
    auto ghosts = [&](int e, int f, double* dst, int64_t stride) {
        const int dd = f >> 1, sd = f & 1;
        const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
        for (int g = 0; g < GH; ++g)
            for (int b = 0; b < nc; ++b)
                for (int aa = 0; aa < nc; ++aa) {
                    double xi[3], x[3], ij[3][3], out[NMET];
                    xi[dd] = sd ? 1.0 + (g + 0.5) * dxi : -(1.0 + (g + 0.5) * dxi);
                    xi[t1] = -1.0 + (aa + 0.5) * dxi;
                    xi[t2] = -1.0 + (b + 0.5) * dxi;
                    map(e, xi, x, ij);
                    ks_point(x, M, a, out);
                    for (int q = 0; q < NPM; ++q) dst[q * stride + (int64_t)g * nc * nc + aa + nc * b] = out[q];
                }
    };
    const int64_t per = (int64_t)NPM * GH * nc * nc;
    if (c->nbf > 0) {
        std::vector<double> mg((size_t)c->nbf * per);
        parallel_for(E, [&](int64_t e) {
            for (int f = 0; f < 6; ++f) {
                const int sl = c->h_bface[6 * e + f];
                if (sl >= 0) ghosts((int)e, f, mg.data() + sl * per, (int64_t)GH * nc * nc);
            }
        });
        double* d_mg;
        if ((s = dalloc(c, &d_mg, mg.size()))) return s;
        CK(cudaMemcpy(d_mg, mg.data(), mg.size() * 8, cudaMemcpyHostToDevice));
        d.metgb = d_mg;
    }
    return FFE_OK;
}

// Faces between cubed-sphere wedges: there the FD ghosts are the neighbour's
// data interpolated to this element's grid continued past the face
// (k_fd_fill_ghosts_interp).  nbr: neighbour of every element face.
ffe_status set_ginterp(ffe_ctx* c, const std::vector<int>& nbr) {
    Dev& d = c->d;
    auto wedge = [&](int e) {
        if (c->batch) {
            const InstInfo& in = c->insts[c->h_einst[e]];
            return (e - in.e0) / (in.na * in.na * in.nr);
        }
        return e / (c->shell.na * c->shell.na * c->shell.nr);
    };
    std::vector<unsigned char> gi(6 * (size_t)d.E, 0);
    bool any = false;
    for (int e = 0; e < d.E; ++e)
        for (int f = 0; f < 6; ++f) {
            const int nb = nbr[6 * (size_t)e + f];
            if (nb >= 0 && wedge(nb) != wedge(e)) {
                gi[6 * (size_t)e + f] = 1;
                any = true;
            }
        }
    c->h_ginterp = gi;
    if (!any) return FFE_OK;
    unsigned char* p;
    ffe_status s;
    if ((s = dalloc(c, &p, gi.size()))) return s;
    CK(cudaMemcpy(p, gi.data(), gi.size(), cudaMemcpyHostToDevice));
    d.ginterp = p;
    // per ghost of those faces: its reference coordinates in the neighbour
    // (closed-form inverse of the neighbour's wedge map) turned into the
    // interpolation data the kernels use -- the first cell and the 6-point
    // Lagrange weights of the stencil through the neighbour's subcell centres
    // along each axis, and the Lagrange weights of its LGL nodes along each
    // axis -- so that the kernels do no transcendental or division work
    std::vector<int> slot(gi.size(), -1);
    int ns = 0;
    for (size_t i = 0; i < gi.size(); ++i)
        if (gi[i]) slot[i] = ns++;
    const int ncm = d.nc, ghn = GH * ncm * ncm;
    std::vector<int> gst((size_t)ns * ghn * 3, 0);
    std::vector<double> gwf((size_t)ns * ghn * 18, 0.0), gwl((size_t)ns * ghn * 3 * MAXNP, 0.0);
    auto geo_of = [&](int e, int& el) {
        if (c->batch) {
            const InstInfo& in = c->insts[c->h_einst[e]];
            el = e - in.e0;
            return ShellGeo{in.r_in, in.c, in.na, in.nr};
        }
        el = e;
        return c->shell;
    };
    parallel_for(d.E, [&](int64_t e) {
        for (int f = 0; f < 6; ++f) {
            const int sl = slot[6 * e + f];
            if (sl < 0) continue;
            const int nb = nbr[6 * (size_t)e + f];
            const int P = host_P(c, (int)e), nc = 2 * P + 1, np1 = P + 1;
            const Tables& T = c->tabs_h[P];
            int el, eln;
            const ShellGeo ge = geo_of((int)e, el), gn = geo_of(nb, eln);
            for (int t = 0; t < GH * nc * nc; ++t) {
                const int g = t / (nc * nc), ta = t % nc, tb = (t / nc) % nc;
                double xn[3];
                shell_ghost_ref(ge, el, gn, eln, f >> 1, f & 1, g, ta, tb, nc, xn);
                const size_t gi3 = ((size_t)sl * ghn + t) * 3;
                for (int a = 0; a < 3; ++a) {
                    gst[gi3 + a] = fd6_stencil(nc, xn[a], &gwf[((size_t)sl * ghn + t) * 18 + 6 * a]);
                    lagrange_at(T.x, np1, xn[a], &gwl[(gi3 + a) * MAXNP]);
                }
            }
        }
    });
    // per slot the box of neighbour cells its stencils cover (first cell and
    // extent along each axis): the kernels stage it in shared memory
    std::vector<int> box((size_t)ns * 6, 0);
    int vmax = 0;
    for (int sl = 0; sl < ns; ++sl) {
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
        for (int t = 0; t < ghn; ++t)
            for (int a = 0; a < 3; ++a) {
                const int v = gst[((size_t)sl * ghn + t) * 3 + a];
                lo[a] = v < lo[a] ? v : lo[a];
                hi[a] = v > hi[a] ? v : hi[a];
            }
        int vol = 1;
        for (int a = 0; a < 3; ++a) {
            box[6 * sl + a] = lo[a];
            box[6 * sl + 3 + a] = hi[a] + 6 - lo[a];
            vol *= hi[a] + 6 - lo[a];
        }
        vmax = vol > vmax ? vol : vmax;
    }
    int *d_sl, *d_st, *d_box;
    double *d_wf, *d_wl;
    if ((s = dalloc(c, &d_box, box.size()))) return s;
    CK(cudaMemcpy(d_box, box.data(), box.size() * sizeof(int), cudaMemcpyHostToDevice));
    d.gbox = d_box;
    d.gbox_max = vmax;
    if ((s = dalloc(c, &d_sl, slot.size()))) return s;
    if ((s = dalloc(c, &d_st, gst.size()))) return s;
    if ((s = dalloc(c, &d_wf, gwf.size()))) return s;
    if ((s = dalloc(c, &d_wl, gwl.size()))) return s;
    CK(cudaMemcpy(d_sl, slot.data(), slot.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_st, gst.data(), gst.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_wf, gwf.data(), gwf.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_wl, gwl.data(), gwl.size() * 8, cudaMemcpyHostToDevice));
    d.gislot = d_sl;
    d.gst = d_st;
    d.gwf = d_wf;
    d.gwl = d_wl;
    c->h_gislot = slot;
    return FFE_OK;
}

// Six-wedge shell: coordinates, per-node inverse Jacobians, connectivity with
// orientation, boundary kinds, Kerr-Schild metric arrays and (dx)_min.
ffe_status build_shell(ffe_ctx* c) {
    const int E = c->d.E, np1 = c->d.np1, nc = c->d.nc, nn = c->d.nn, ncell = c->d.ncell;
    const int64_t ndg = c->d.ndg, nfd = c->d.nfd;
    MapFn map = ctx_map(c);
    std::vector<double> xdg(3 * (size_t)ndg), xfd(3 * (size_t)nfd), geo(9 * (size_t)ndg);
    parallel_for(E, [&](int64_t e) {
        for (int q = 0; q < nn; ++q) {
            const int i = q % np1, j = (q / np1) % np1, k = q / (np1 * np1);
            const double xi[3] = {c->tab.x[i], c->tab.x[j], c->tab.x[k]};
            double x[3], ij[3][3];
            map((int)e, xi, x, ij);
            const int64_t p = e * nn + q;
            for (int a = 0; a < 3; ++a) xdg[a * ndg + p] = x[a];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) geo[(3 * a + b) * ndg + p] = ij[a][b];
        }
        for (int q = 0; q < ncell; ++q) {
            const int cc[3] = {q % nc, (q / nc) % nc, q / (nc * nc)};
            double xi[3], x[3], ij[3][3];
            for (int a = 0; a < 3; ++a) xi[a] = -1.0 + (cc[a] + 0.5) * 2.0 / nc;
            map((int)e, xi, x, ij);
            for (int a = 0; a < 3; ++a) xfd[a * nfd + e * ncell + q] = x[a];
        }
    });
    std::vector<double> xn(c->tab.x, c->tab.x + np1);
    std::vector<int> nbr, nbf, orient, bc(6 * E, 0), bface(6 * E, -1);
    match_faces(E, map, xn, np1, c->dom.r_out, nbr, nbf, orient);
    int nbfd = 0;
    for (int e = 0; e < E; ++e)
        for (int f = 0; f < 6; ++f) {
            if (nbr[6 * e + f] == -2) return fail(FFE_EINVAL, "no orientation matches face %d of element %d", f, e);
            if (nbr[6 * e + f] >= 0) continue;
            int ia, ib, ir, w;
            shell_elem(c->shell, e, ia, ib, ir, w);
            int kind;
            if (f == 4 && ir == 0) kind = c->dom.bc_lo[0];
            else if (f == 5 && ir == c->shell.nr - 1) kind = c->dom.bc_hi[0];
            else return fail(FFE_EINVAL, "unmatched interior face %d of element %d", f, e);
            if (kind == FFE_BC_PERIODIC) return fail(FFE_EINVAL, "a shell has no periodic boundary");
            bc[6 * e + f] = kind;
            if (kind == FFE_BC_DIRICHLET) bface[6 * e + f] = nbfd++;
        }
    c->nbf = nbfd;
    c->h_bface = bface;
    if (ffe_status sg = set_ginterp(c, nbr)) return sg;
    // (dx)_min along element grid lines
    double dmin = 1e300;
    for (int64_t e = 0; e < E; ++e)
        for (int q = 0; q < nn; ++q) {
            const int ci[3] = {q % np1, (q / np1) % np1, q / (np1 * np1)};
            for (int a = 0; a < 3; ++a) {
                if (ci[a] == np1 - 1) continue;
                const int q2 = q + (a == 0 ? 1 : (a == 1 ? np1 : np1 * np1));
                double s2 = 0.0;
                for (int b = 0; b < 3; ++b) {
                    const double dx = xdg[b * ndg + e * nn + q2] - xdg[b * ndg + e * nn + q];
                    s2 += dx * dx;
                }
                dmin = fmin(dmin, sqrt(s2));
            }
        }
    c->dxmin = dmin;
    ffe_status s;
    double *d_xdg, *d_xfd, *d_geo, *d_bdg, *d_bfd, *d_ijac;
    int *d_nbr, *d_nbf, *d_bc, *d_bface, *d_or;
    if ((s = dalloc(c, &d_xdg, xdg.size()))) return s;
    if ((s = dalloc(c, &d_xfd, xfd.size()))) return s;
    if ((s = dalloc(c, &d_geo, geo.size()))) return s;
    if ((s = dalloc(c, &d_ijac, 3 * (size_t)E))) return s;
    if ((s = dalloc(c, &d_nbr, nbr.size()))) return s;
    if ((s = dalloc(c, &d_nbf, nbf.size()))) return s;
    if ((s = dalloc(c, &d_or, orient.size()))) return s;
    if ((s = dalloc(c, &d_bc, bc.size()))) return s;
    if ((s = dalloc(c, &d_bface, bface.size()))) return s;
    if ((s = dalloc(c, &d_bdg, (size_t)(nbfd > 0 ? nbfd : 1) * NV * np1 * np1))) return s;
    if ((s = dalloc(c, &d_bfd, (size_t)(nbfd > 0 ? nbfd : 1) * NV * GH * nc * nc))) return s;
    CK(cudaMemcpy(d_xdg, xdg.data(), xdg.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_xfd, xfd.data(), xfd.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_nbf, nbf.data(), nbf.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_or, orient.data(), orient.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_bc, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_bface, bface.data(), bface.size() * 4, cudaMemcpyHostToDevice));
    Dev& d = c->d;
    d.xyz_dg = d_xdg;
    d.xyz_fd = d_xfd;
    d.xfd_n = (int64_t)d.E * d.ncell;
    d.geo = d_geo;
    d.ijac = d_ijac;
    d.nbr = d_nbr;
    d.nbr_face = d_nbf;
    d.orient = d_or;
    d.bc = d_bc;
    d.bface = d_bface;
    d.bdg = d_bdg;
    d.bfd = d_bfd;
    d.curved = 1;
    d.shell_rin = c->shell.r_in;
    d.shell_c = c->shell.c;
    d.shell_na = c->shell.na;
    d.shell_nr = c->shell.nr;
    if (c->met.kind == FFE_METRIC_KERR_SCHILD) {
        std::vector<double> met((size_t)NMET * ndg);
        std::vector<double> lam(ndg);
        const double M = c->met.M, a = c->met.a;
        parallel_for(ndg, [&](int64_t p) {
            double x[3] = {xdg[p], xdg[ndg + p], xdg[2 * ndg + p]}, out[NMET];
            ks_point(x, M, a, out);
            for (int q = 0; q < NMET; ++q) met[q * ndg + p] = out[q];
            // alpha + |beta|_gamma
            const double* gl = out + M_GL;
            const double* b = out + M_BETA;
            const double bb = gl[0] * b[0] * b[0] + gl[3] * b[1] * b[1] + gl[5] * b[2] * b[2] +
                              2.0 * (gl[1] * b[0] * b[1] + gl[2] * b[0] * b[2] + gl[4] * b[1] * b[2]);
            lam[p] = out[M_ALPHA] + sqrt(bb);
        });
        double* d_met;
        if ((s = dalloc(c, &d_met, met.size()))) return s;
        CK(cudaMemcpy(d_met, met.data(), met.size() * 8, cudaMemcpyHostToDevice));
        d.met = d_met;
        d.ks = 1;
        c->lam_max = 0.0;
        for (double v : lam) c->lam_max = fmax(c->lam_max, v);
        if (c->prm.tci_on && (s = build_ks_fd_tables(c, xfd))) return s;
    }
    return FFE_OK;
}

// Dirichlet boundary data = the initial data at face nodes and ghost-cell centres.
ffe_status fill_dirichlet(ffe_ctx* c) {
    if (c->nbf == 0) return FFE_OK;
    const int np1m = c->d.np1, ncm = c->d.nc, E = c->d.E;
    std::vector<double> bdg((size_t)c->nbf * NV * np1m * np1m), bfd((size_t)c->nbf * NV * GH * ncm * ncm);
    MapFn map = ctx_map(c);
    for (int e = 0; e < E; ++e) {
        const int P = host_P(c, e), np1 = P + 1, nc = 2 * P + 1;
        const Tables& T = c->tabs_h[P];
        const double* prm = c->batch ? c->id_prm_inst.data() + (size_t)c->h_einst[e] * c->id_nprm : c->id_prm.data();
        const int nprm = c->batch ? c->id_nprm : (int)c->id_prm.size();
        for (int f = 0; f < 6; ++f) {
            const int slot = c->h_bface[6 * e + f];
            if (slot < 0) continue;
            const int dd = f >> 1, s = f & 1;
            const int t1 = dd == 0 ? 1 : 0, t2 = dd == 2 ? 1 : 2;
            for (int b = 0; b < np1; ++b)
                for (int a = 0; a < np1; ++a) {
                    double xi[3];
                    xi[dd] = s ? 1.0 : -1.0;
                    xi[t1] = T.x[a];
                    xi[t2] = T.x[b];
                    double X[3], U[NV], ij[3][3];
                    map(e, xi, X, ij);
                    initial_point(c->id_kind, prm, nprm, X, U);
                    for (int v = 0; v < NV; ++v) bdg[((size_t)slot * NV + v) * np1m * np1m + a + np1 * b] = U[v];
                }
            for (int g = 0; g < GH; ++g)
                for (int b = 0; b < nc; ++b)
                    for (int a = 0; a < nc; ++a) {
                        double xi[3];
                        const double dxi = 2.0 / nc;
                        xi[dd] = s ? 1.0 + (g + 0.5) * dxi : -(1.0 + (g + 0.5) * dxi);
                        xi[t1] = -1.0 + (a + 0.5) * dxi;
                        xi[t2] = -1.0 + (b + 0.5) * dxi;
                        double X[3], U[NV], ij[3][3];
                        map(e, xi, X, ij);
                        initial_point(c->id_kind, prm, nprm, X, U);
                        for (int v = 0; v < NV; ++v)
                            bfd[(((size_t)slot * NV + v) * GH + g) * ncm * ncm + a + nc * b] = U[v];
                    }
        }
    }
    CK(cudaMemcpy((void*)c->d.bdg, bdg.data(), bdg.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)c->d.bfd, bfd.data(), bfd.size() * 8, cudaMemcpyHostToDevice));
    return FFE_OK;
}

// One IMEX-SSP3(4,3,3) step with the hybrid control loop, enqueued on c->st.
void enqueue_step(ffe_ctx* c) {
    const Dev& d = c->d;
    cudaStream_t st = c->st;
    cudaMemsetAsync(d.counts + 2, 0, 2 * sizeof(int), st);
    cudaMemsetAsync(d.switched, 0, d.E, st);
    launch_build_lists(d, st);
    if (d.ks) launch_stage12_ks(d, c->un, c->Ua, c->G1, c->G2, st);
    else launch_stage12(d, c->un, c->Ua, c->G1, c->G2, st);
    struct S { int sub; Field Uin, Fout, Uout, Gout; };
    const S subs[3] = {{SUB_A, c->Ua, c->F2, c->Ub, c->G3},
                       {SUB_B, c->Ub, c->F3, c->Ua, c->G4},
                       {SUB_C, c->Ua, c->Fs, c->un, c->G4}};
    for (const S& s : subs) {
        if (!d.ks || d.metfd) launch_current(d, s.Uin, c->J, nullptr, 0, st);
        if (d.curved)
            launch_dg_substep_curved(d, s.sub, s.Uin, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, s.Fout,
                                     s.Uout, s.Gout, st);
        else
            launch_dg_substep(d, s.sub, s.Uin, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, s.Fout,
                              s.Uout, s.Gout, st);
        launch_fd_substep(d, s.sub, d.fd_list, 1, s.Uin, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4,
                          s.Fout, s.Uout, s.Gout, st);
        if (d.tci_on) {
            launch_rollback_project(d, s.sub, c->un, s.Uin, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, st);
            launch_current(d, s.Uin, c->J, d.flag_list, 2, st);
            launch_fd_substep(d, s.sub, d.flag_list, 2, s.Uin, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3,
                              c->G4, s.Fout, s.Uout, s.Gout, st);
            cudaMemsetAsync(d.counts + 2, 0, sizeof(int), st);
            launch_build_lists(d, st);
        }
    }
    if (d.tci_on) launch_fd2dg(d, c->un, st);
}

// Launch-shape autotuner: times the DG right-hand side (no state change) with
// persistent grids of 1, 2, 3, 4, 6 and 8 CTAs per SM and keeps the fastest,
// for the highest order and, in a batch, separately for the elements of each
// lower order (each order runs its own kernel in CTAs sized for it, so each
// has its own best grid: elements per CTA per order).  The whole right-hand
// side is timed each time, one order's grid varied, the others at their best
// so far.
ffe_status autotune(ffe_ctx* c) {
    Dev& d = c->d;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch_build_lists(d, c->st);
    if (!d.ks || d.metfd) launch_current(d, c->un, c->J, nullptr, 0, c->st);
    int* slots[3] = {&d.dg_grid, &d.dg_grid_lo, &d.dg_grid_lo2};
    const int nord = c->batch ? 3 : 1;
    for (int o = 0; o < nord; ++o) {
        if (o == 1 && !d.dg_list_lo) continue;
        if (o == 2 && !d.dg_list_lo2) continue;
        float best = 1e30f;
        int best_g = 0;
        for (int k : {1, 2, 3, 4, 6, 8}) {
            *slots[o] = k * d.nsm;
            float tot = 0.0f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaEventRecord(a, c->st));
                if (d.curved)
                    launch_dg_substep_curved(d, SUB_RHS, c->un, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4,
                                             c->Fs, c->Fs, c->G1, c->st);
                else
                    launch_dg_substep(d, SUB_RHS, c->un, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, c->Fs,
                                      c->Fs, c->G1, c->st);
                CK(cudaEventRecord(b, c->st));
                CK(cudaEventSynchronize(b));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (rep > 0) tot += ms;
            }
            if (tot < best) { best = tot; best_g = k * d.nsm; }
        }
        *slots[o] = best_g;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->tuned = true;
    return FFE_OK;
}

ffe_status run_steps(ffe_ctx* c, int nsteps) {
    static const bool no_graph = getenv("FFE_NO_GRAPH") != nullptr;
    if (!c->tuned && nsteps > 0 && getenv("FFE_NO_AUTOTUNE") == nullptr) {
        ffe_status s = autotune(c);
        if (s) return s;
    }
    for (int n = 0; n < nsteps; ++n) {
        if (g_prof.on) {
            enqueue_step(c);
            prof_collect(c->st);
            CK(cudaGetLastError());
            c->t += c->d.dt;
            c->steps += 1;
            continue;
        }
        if (!no_graph && c->graph_ok && c->gexec == nullptr && c->steps > 0) {
            // capture one step (kernels were launched eagerly once, so attributes are set)
            cudaGraph_t g;
            if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                enqueue_step(c);
                if (cudaStreamEndCapture(c->st, &g) == cudaSuccess &&
                    cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess) {
                    c->graph = g;
                    size_t nn = 0;
                    cudaGraphGetNodes(g, nullptr, &nn);
                    std::vector<cudaGraphNode_t> nodes(nn);
                    cudaGraphGetNodes(g, nodes.data(), &nn);
                    c->graph_kernels = 0;
                    for (auto& nd : nodes) {
                        cudaGraphNodeType ty;
                        cudaGraphNodeGetType(nd, &ty);
                        c->graph_kernels += ty == cudaGraphNodeTypeKernel;
                    }
                } else {
                    c->graph_ok = false;
                    c->gexec = nullptr;
                    cudaGetLastError();
                }
            } else {
                c->graph_ok = false;
                cudaGetLastError();
            }
        }
        if (c->gexec) {
            CK(cudaGraphLaunch(c->gexec, c->st));
            g_launch_counter += c->graph_kernels;
        } else {
            enqueue_step(c);
        }
        CK(cudaGetLastError());
        c->t += c->d.dt;
        c->steps += 1;
    }
    return FFE_OK;
}

// Tables for every order in use, thresholds, per-element arrays, work buffers
// and the FD slot pool.  d.P/np1/nn/nc/ncell already hold the largest order's
// sizes and d.E the element count; fd_cap the number of FD slots.
ffe_status finish_create(ffe_ctx* c, int fd_cap, const std::vector<int>& orders) {
    Dev& d = c->d;
    const ffe_params* params = &c->prm;
    ffe_status s;
    for (int P : orders) {
        build_tables(P, params->filter_a, params->filter_b, params->tci_M, c->tabs_h[P]);
        d.thr_dgP[P] = pow((double)(P + 1 - params->tci_M), -params->tci_alpha);
        d.thr_fdP[P] = pow((double)(P + 1 - params->tci_M), -(params->tci_alpha + 1.0));
    }
    c->tab = c->tabs_h[d.P];
    Tables* dtabs;
    if ((s = dalloc(c, &dtabs, MAXNP))) return s;
    CK(cudaMemcpy(dtabs, c->tabs_h, sizeof(c->tabs_h), cudaMemcpyHostToDevice));
    d.tabs = dtabs;
    d.tab = dtabs + d.P;
    d.thr_dg = d.thr_dgP[d.P];
    d.thr_fd = d.thr_fdP[d.P];
    d.fd_cap = fd_cap;
    d.nfd = (int64_t)fd_cap * d.ncell;
    const int chunk = params->fd_chunk > 0 ? params->fd_chunk : 2048;
    d.chunk = fd_cap < chunk ? (fd_cap > 0 ? fd_cap : 1) : chunk;
    if ((s = dalloc(c, &d.mask, d.E))) return s;
    if ((s = dalloc(c, &d.switched, d.E))) return s;
    if ((s = dalloc(c, &d.dg_list, d.E))) return s;
    if ((s = dalloc(c, &d.fd_list, d.E))) return s;
    if ((s = dalloc(c, &d.flag_list, d.E))) return s;
    if ((s = dalloc(c, &d.near_list, 4096))) return s;
    if ((s = dalloc(c, &d.counts, 8))) return s;
    if ((s = dalloc(c, &d.units, 3))) return s;   // node updates, FD and DG element updates
    if (d.curved) {
        // FD-point tables of the shell map (Dev::stab): gnomonic coordinate
        // X = tan(pi/4 e) and 1/(pi/4 (1 + X^2)) on the half-cell grid of the
        // angular rows, r and 1/r on that of the radial rows
        std::vector<double> tab;
        auto add = [&](int P, int na, int nr, double r_in, double cc) {
            const int off = (int)tab.size(), nc = 2 * P + 1;
            const long double q = 0.785398163397448309615660845819875721L;
            std::vector<double> X(2 * nc * na + 1), R(2 * nc * nr + 1);
            for (size_t g = 0; g < X.size(); ++g) X[g] = (double)std::tan(q * (-1.0L + (long double)g / (nc * na)));
            for (size_t g = 0; g < R.size(); ++g) R[g] = (double)(r_in * std::exp((long double)cc * g / (nc * nr)));
            for (double x : X) tab.push_back(x);
            for (double x : X) tab.push_back((double)(1.0L / (q * (1.0L + (long double)x * x))));
            for (double r : R) tab.push_back(r);
            for (double r : R) tab.push_back(1.0 / r);
            return off;
        };
        if (c->batch)
            for (auto& in : c->insts) in.tab = add(in.P, in.na, in.nr, in.r_in, in.c);
        else
            add(d.P, c->shell.na, c->shell.nr, c->shell.r_in, c->shell.c);
        double* dt;
        if ((s = dalloc(c, &dt, tab.size()))) return s;
        CK(cudaMemcpy(dt, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
        d.stab = dt;
    }
    if (c->batch) {
        int *eP8, *ein;
        InstInfo* dinst;
        std::vector<unsigned char> ep(c->h_eP.begin(), c->h_eP.end());
        unsigned char* dep;
        if ((s = dalloc(c, &dep, d.E))) return s;
        if ((s = dalloc(c, &ein, d.E))) return s;
        if ((s = dalloc(c, &dinst, c->insts.size()))) return s;
        CK(cudaMemcpy(dep, ep.data(), d.E, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ein, c->h_einst.data(), d.E * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dinst, c->insts.data(), c->insts.size() * sizeof(InstInfo), cudaMemcpyHostToDevice));
        d.eP = dep;
        d.einst = ein;
        d.inst = dinst;
        (void)eP8;
        // DG elements of the lower orders get their own work lists (own launches)
        if ((s = dalloc(c, &d.dg_list_lo, d.E))) return s;
        if ((s = dalloc(c, &d.dg_list_lo2, d.E))) return s;
    }
    if (c->batch || fd_cap < d.E) {
        // FD slot pool: every slot free until ffe_set_initial assigns some
        if ((s = dalloc(c, &d.fd_slot, d.E))) return s;
        if ((s = dalloc(c, &d.slot_elem, fd_cap))) return s;
        if ((s = dalloc(c, &d.free_slots, fd_cap))) return s;
    }
    for (Field* f : {&c->un, &c->Ua, &c->Ub, &c->F2, &c->F3, &c->Fs})
        if ((s = alloc_field(c, *f, NV))) return s;
    for (Field* f : {&c->G1, &c->G2, &c->G3, &c->G4})
        if ((s = alloc_field(c, *f, NG))) return s;
    if ((s = alloc_field(c, c->J, NJ))) return s;
    const int64_t ne = d.nc + 2 * GH;
    if ((s = dalloc(c, &d.ext, (size_t)12 * d.chunk * ne * ne * ne))) return s;
    if ((s = dalloc(c, &d.flux, (size_t)(d.curved ? 9 : 3) * NV * d.chunk * (d.nc + 1) * d.nc * d.nc))) return s;
    if ((s = dalloc(c, &d.ftr, (size_t)fd_cap * 6 * 12 * d.np1 * d.np1))) return s;
    return FFE_OK;
}

// Assign FD slots to the elements flagged at initialisation (pool contexts).
ffe_status init_slots(ffe_ctx* c, const std::vector<unsigned char>& mask) {
    Dev& d = c->d;
    if (!d.fd_slot) return FFE_OK;
    std::vector<int> slot(d.E, -1), selem(d.fd_cap, -1), freel;
    int next = 0;
    for (int e = 0; e < d.E; ++e)
        if (mask[e]) {
            if (next >= d.fd_cap)
                return fail(FFE_ENOMEM, "the initial data put more than fd_capacity = %d elements on FD", d.fd_cap);
            slot[e] = next;
            selem[next] = e;
            ++next;
        }
    for (int sl = d.fd_cap - 1; sl >= next; --sl) freel.push_back(sl);
    freel.resize(d.fd_cap, -1);
    const int nfree = d.fd_cap - next;
    CK(cudaMemcpy(d.fd_slot, slot.data(), d.E * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.slot_elem, selem.data(), d.fd_cap * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.free_slots, freel.data(), d.fd_cap * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.counts + 5, &nfree, sizeof(int), cudaMemcpyHostToDevice));
    c->h_fd_slot = slot;
    return FFE_OK;
}

// Initial data for all elements (per-instance parameters in batched contexts).
ffe_status set_initial_impl(ffe_ctx* c, int id_kind, bool keep_mask, bool via_fd) {
    const Dev& d = c->d;
    auto prm_of = [&](int e) -> const double* {
        return c->batch ? c->id_prm_inst.data() + (size_t)c->h_einst[e] * c->id_nprm : c->id_prm.data();
    };
    const int nprm = c->batch ? c->id_nprm : (int)c->id_prm.size();
    std::vector<double> xdg(3 * (size_t)d.ndg), U(NV * (size_t)(d.ndg + d.nfd), 0.0);
    CK(cudaMemcpy(xdg.data(), d.xyz_dg, xdg.size() * 8, cudaMemcpyDeviceToHost));
    parallel_for(d.ndg, [&](int64_t p) {
        const int e = (int)(p / d.nn);
        const int P = host_P(c, e);
        if ((int)(p % d.nn) >= (P + 1) * (P + 1) * (P + 1)) return;
        double X[3] = {xdg[p], xdg[d.ndg + p], xdg[2 * d.ndg + p]}, u[NV];
        initial_point(id_kind, prm_of(e), nprm, X, u);
        for (int v = 0; v < NV; ++v) U[v * d.ndg + p] = u[v];
    });
    std::vector<unsigned char> mask(d.E, via_fd ? 1 : 0);
    if (keep_mask) CK(cudaMemcpy(mask.data(), d.mask, d.E, cudaMemcpyDeviceToHost));
    if (d.tci_on || keep_mask || via_fd) {
        ffe_status s;
        if (!keep_mask && !via_fd) {
            double* ratio;
            if ((s = dalloc(c, &ratio, d.E))) return s;
            CK(cudaMemcpy(c->un.p, U.data(), NV * d.ndg * 8, cudaMemcpyHostToDevice));
            launch_tci_ratio(d, c->un.p, ratio, c->st);
            std::vector<double> r(d.E);
            CK(cudaMemcpyAsync(r.data(), ratio, d.E * 8, cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            for (int e = 0; e < d.E; ++e) mask[e] = r[e] > d.thr_dgP[host_P(c, e)];
        }
        if ((s = init_slots(c, mask))) return s;
        MapFn map = ctx_map(c);
        parallel_for(d.E, [&](int64_t e) {
            if (!mask[e]) return;
            const int P = host_P(c, (int)e), nc = 2 * P + 1;
            const int64_t base = (int64_t)(d.fd_slot ? c->h_fd_slot[e] : e) * d.ncell;
            for (int q = 0; q < nc * nc * nc; ++q) {
                const int cc[3] = {q % nc, (q / nc) % nc, q / (nc * nc)};
                double xi[3], X[3], ij[3][3], u[NV];
                for (int a = 0; a < 3; ++a) xi[a] = -1.0 + (cc[a] + 0.5) * 2.0 / nc;
                map((int)e, xi, X, ij);
                initial_point(id_kind, prm_of((int)e), nprm, X, u);
                for (int v = 0; v < NV; ++v) U[NV * d.ndg + v * d.nfd + base + q] = u[v];
            }
        });
    }
    CK(cudaMemcpy(c->un.p, U.data(), U.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.mask, mask.data(), d.E, cudaMemcpyHostToDevice));
    ffe_status s;
    if ((s = fill_dirichlet(c))) return s;
    CK(cudaMemset(d.units, 0, 3 * sizeof(unsigned long long)));
    c->t = 0.0;
    c->steps = 0;
    c->ref_valid = false;
    return FFE_OK;
}


// The analytic initial data of the context at the DG nodes of its DG elements
// and the subcells of its FD elements (state-vector layout, in d_ref): the
// exact solution of a stationary problem such as the Wald field.  Rebuilt
// when the mask, the FD slots or the initial data changed since the last build.
ffe_status build_reference(ffe_ctx* c) {
    const Dev& d = c->d;
    std::vector<unsigned char> mask(d.E);
    std::vector<int> slot;
    CK(cudaMemcpyAsync(mask.data(), d.mask, d.E, cudaMemcpyDeviceToHost, c->st));
    if (d.fd_slot) {
        slot.resize(d.E);
        CK(cudaMemcpyAsync(slot.data(), d.fd_slot, d.E * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    if (c->ref_valid && mask == c->ref_mask && slot == c->ref_slot) return FFE_OK;
    ffe_status s;
    const size_t n = (size_t)NV * (d.ndg + d.nfd);
    if (!c->d_ref && (s = dalloc(c, &c->d_ref, n))) return s;
    auto prm_of = [&](int e) -> const double* {
        return c->batch ? c->id_prm_inst.data() + (size_t)c->h_einst[e] * c->id_nprm : c->id_prm.data();
    };
    const int nprm = c->batch ? c->id_nprm : (int)c->id_prm.size();
    std::vector<double> xdg(3 * (size_t)d.ndg), R(n, 0.0);
    CK(cudaMemcpy(xdg.data(), d.xyz_dg, xdg.size() * 8, cudaMemcpyDeviceToHost));
    parallel_for(d.ndg, [&](int64_t p) {
        const int e = (int)(p / d.nn);
        const int P = host_P(c, e);
        if (mask[e] || (int)(p % d.nn) >= (P + 1) * (P + 1) * (P + 1)) return;
        double X[3] = {xdg[p], xdg[d.ndg + p], xdg[2 * d.ndg + p]}, u[NV];
        initial_point(c->id_kind, prm_of(e), nprm, X, u);
        for (int v = 0; v < NV; ++v) R[v * d.ndg + p] = u[v];
    });
    MapFn map = ctx_map(c);
    parallel_for(d.E, [&](int64_t e) {
        if (!mask[e]) return;
        const int P = host_P(c, (int)e), nc = 2 * P + 1;
        const int64_t base = (int64_t)(d.fd_slot ? slot[e] : e) * d.ncell;
        if (base < 0) return;
        for (int q = 0; q < nc * nc * nc; ++q) {
            const int cc[3] = {q % nc, (q / nc) % nc, q / (nc * nc)};
            double xi[3], X[3], ij[3][3], u[NV];
            for (int a = 0; a < 3; ++a) xi[a] = -1.0 + (cc[a] + 0.5) * 2.0 / nc;
            map((int)e, xi, X, ij);
            initial_point(c->id_kind, prm_of((int)e), nprm, X, u);
            for (int v = 0; v < NV; ++v) R[NV * d.ndg + v * d.nfd + base + q] = u[v];
        }
    });
    CK(cudaMemcpy(c->d_ref, R.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    c->ref_mask = mask;
    c->ref_slot = slot;
    c->ref_valid = true;
    return FFE_OK;
}


// Surface quadrature on the shell's coordinate surface of radius r (the sphere
// |x| = r; on a spherical Kerr-Schild shell the spheroid of Kerr-Schild radius
// r) -- the luminosity of Sec. IV.C.2 and the horizon flux of Sec. IV.B.2: the
// radial element layer that contains r, the Lagrange weights lk[np1] of xi^3
// at r (closed-form inverse of the logarithmic radial map), and per surface
// node (i, j) of each element of the layer the LGL weights times the exact
// area element and the outward unit normal, wn[4] = (w_i w_j |a1 x a2|,
// (a1 x a2)/|a1 x a2|), a_k = dx/dxi^k (on a sphere the normal is r^).  upper:
// only the elements whose centre has z > 0 (the equator must then lie on
// element boundaries).  inst >= 0: the shell of that instance of a batch (its
// elements e0 .. e0 + 6 na^2 nr - 1, at the batch's top order).
void surface_setup(ffe_ctx* c, double r, bool upper, int inst, std::vector<int>& elem, std::vector<double>& lk,
                   std::vector<double>& wn) {
    const Dev& d = c->d;
    ShellGeo g = c->shell;
    int e0 = 0, ne = d.E;
    const Tables* tb = &c->tab;
    if (inst >= 0) {
        const InstInfo& in = c->insts[inst];
        g = ShellGeo{in.r_in, in.c, in.na, in.nr};
        e0 = in.e0;
        ne = 6 * in.na * in.na * in.nr;
        tb = &c->tabs_h[in.P];
    }
    const Tables& T = *tb;
    const double er = std::log(r / g.r_in) / g.c - 1.0;
    const double pos = (er + 1.0) / 2.0 * g.nr;
    int ir = (int)std::floor(pos);
    ir = ir > g.nr - 1 ? g.nr - 1 : ir;
    const double xr = 2.0 * (pos - ir) - 1.0;
    const int np1 = d.np1;
    lk.assign(np1, 0.0);
    for (int k = 0; k < np1; ++k) {
        double v = 1.0;
        for (int m = 0; m < np1; ++m)
            if (m != k) v *= (xr - T.x[m]) / (T.x[k] - T.x[m]);
        lk[k] = v;
    }
    for (int e = 0; e < ne; ++e) {
        int ia, ib, irr, w;
        shell_elem(g, e, ia, ib, irr, w);
        if (irr != ir) continue;
        if (upper) {
            const double xi0[3] = {0.0, 0.0, xr};
            double x0[3], ij0[3][3];
            shell_map(g, e, xi0, x0, ij0);
            if (!(x0[2] > 0.0)) continue;
        }
        elem.push_back(e0 + e);
        for (int j = 0; j < np1; ++j)
            for (int i = 0; i < np1; ++i) {
                const double xi[3] = {T.x[i], T.x[j], xr};
                double x[3], ij[3][3];
                shell_map(g, e, xi, x, ij);
                // area element |dx/dxi1 x dx/dxi2| from the Jacobian (inverse of ij)
                double J[3][3];
                const double det = ij[0][0] * (ij[1][1] * ij[2][2] - ij[1][2] * ij[2][1]) -
                                   ij[0][1] * (ij[1][0] * ij[2][2] - ij[1][2] * ij[2][0]) +
                                   ij[0][2] * (ij[1][0] * ij[2][1] - ij[1][1] * ij[2][0]);
                J[0][0] = (ij[1][1] * ij[2][2] - ij[1][2] * ij[2][1]) / det;
                J[0][1] = (ij[0][2] * ij[2][1] - ij[0][1] * ij[2][2]) / det;
                J[1][0] = (ij[1][2] * ij[2][0] - ij[1][0] * ij[2][2]) / det;
                J[1][1] = (ij[0][0] * ij[2][2] - ij[0][2] * ij[2][0]) / det;
                J[2][0] = (ij[1][0] * ij[2][1] - ij[1][1] * ij[2][0]) / det;
                J[2][1] = (ij[0][1] * ij[2][0] - ij[0][0] * ij[2][1]) / det;
                const double a1[3] = {J[0][0], J[1][0], J[2][0]}, a2[3] = {J[0][1], J[1][1], J[2][1]};
                const double cr[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
                // a1 x a2 points to increasing xi^3 (outward) where the map keeps
                // orientation (det > 0); flip it otherwise
                const double area = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
                const double sg = det > 0.0 ? 1.0 : -1.0;
                wn.push_back(T.w[i] * T.w[j] * area);
                wn.push_back(sg * cr[0] / area);
                wn.push_back(sg * cr[1] / area);
                wn.push_back(sg * cr[2] / area);
            }
    }
}

// The quadrature of surface_setup on the device, built once per (r, upper, inst).
ffe_status surface_get(ffe_ctx* c, double r, bool upper, int inst, const ffe_ctx::Surf** out) {
    const auto key = std::make_tuple(r, upper ? 1 : 0, inst);
    auto it = c->surf.find(key);
    if (it == c->surf.end()) {
        std::vector<int> elem;
        std::vector<double> lk, wn;
        surface_setup(c, r, upper, inst, elem, lk, wn);
        ffe_ctx::Surf sf;
        ffe_status s;
        if ((s = dalloc(c, &sf.elem, elem.size()))) return s;
        if ((s = dalloc(c, &sf.lk, lk.size()))) return s;
        if ((s = dalloc(c, &sf.w, wn.size()))) return s;
        CK(cudaMemcpy(sf.elem, elem.data(), elem.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(sf.lk, lk.data(), lk.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(sf.w, wn.data(), wn.size() * 8, cudaMemcpyHostToDevice));
        sf.ns = (int)elem.size();
        it = c->surf.emplace(key, sf).first;
    }
    *out = &it->second;
    return FFE_OK;
}

// Sum of the surface integrand (bflux = 1: B~.n, else (E~ x B~).n) of U over
// sf, into *out_host when it is not NULL (synchronising the context stream);
// grad_dev (may be NULL) receives scale * d(sum)/dU.
ffe_status surface_sum(ffe_ctx* c, const ffe_ctx::Surf& sf, const double* U_dev, int bflux, double* grad_dev,
                       double scale, double* out_host) {
    const Dev& d = c->d;
    ffe_status s;
    if (!c->d_partial && (s = dalloc(c, &c->d_partial, 1024))) return s;
    Field U{(double*)U_dev, NV, d.ndg, d.nfd}, G{grad_dev, NV, d.ndg, d.nfd};
    const int nb = d.nsm;
    launch_luminosity(d, U, sf.elem, sf.lk, sf.w, sf.ns, c->d_partial, nb, G, scale, c->st, bflux);
    if (out_host) {
        std::vector<double> part(nb);
        CK(cudaMemcpyAsync(part.data(), c->d_partial, nb * 8, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        double sum = 0.0;
        for (double v : part) sum += v;
        *out_host = sum;
    }
    CK(cudaGetLastError());
    return FFE_OK;
}

// The shell a surface diagnostic integrates over: the context's, or with a
// batch the instance args[1] (an integer index, required), which must run at
// the batch's top order; r must lie strictly inside that shell.
ffe_status surface_target(ffe_ctx* c, const double* args, double r, int* inst, int* na) {
    const Dev& d = c->d;
    if (!d.curved || (!c->batch && c->dom.kind != FFE_DOMAIN_SHELL6))
        return fail(FFE_ENOTIMPL, "surface diagnostics need a shell");
    double r_in = c->dom.r_in, r_out = c->dom.r_out;
    *inst = -1;
    *na = c->shell.na;
    if (c->batch) {
        const double a1 = args[1];
        if (!(a1 >= 0 && a1 < (double)c->insts.size()) || a1 != std::floor(a1))
            return fail(FFE_EINVAL, "a batched context needs args[1] = an instance index in [0, %d)", (int)c->insts.size());
        const InstInfo& in = c->insts[(int)a1];
        if (in.P != d.P) return fail(FFE_ENOTIMPL, "surface diagnostics of instances below the batch's top order P = %d", d.P);
        *inst = (int)a1;
        *na = in.na;
        r_in = in.r_in;
        r_out = in.r_in * std::exp(2.0 * in.c);
    }
    if (!(r > r_in && r < r_out)) return fail(FFE_EINVAL, "radius %g outside the shell (%g, %g)", r, r_in, r_out);
    return FFE_OK;
}

}  // namespace


namespace ffe {
// error message for entry points defined in other translation units
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace ffe

// ------------------------------------------------------------------ C ABI ---
extern "C" {

// ---- checkpoint / resume ---------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];                    // "FFECKPT1"
    int64_t E, ndg, nfd, fd_cap, n_inst;
    int64_t steps, id_kind, id_nprm_total;
    double t;
    unsigned long long units[3];
    int64_t free_count;
};

size_t ckpt_size(const ffe_ctx* c) {
    const Dev& d = c->d;
    const size_t nprm = c->batch ? c->id_prm_inst.size() : c->id_prm.size();
    size_t b = sizeof(CkptHeader) + nprm * sizeof(double) + NV * (size_t)(d.ndg + d.nfd) * sizeof(double) + d.E;
    if (d.fd_slot) b += sizeof(int) * ((size_t)d.E + 2 * (size_t)d.fd_cap);
    return b;
}
}  // namespace

ffe_status ffe_save(ffe_ctx* c, void* host_buf, size_t* bytes) try {
    g_err.clear();
    if (!c || !bytes) return fail(FFE_EINVAL, "null argument");
    const Dev& d = c->d;
    const size_t need = ckpt_size(c);
    if (!host_buf) {
        *bytes = need;
        return FFE_OK;
    }
    if (*bytes < need) return fail(FFE_EINVAL, "checkpoint buffer of %zu bytes, %zu needed", *bytes, need);
    if (c->id_kind < 0) return fail(FFE_ESTATE, "no initial data set");
    CkptHeader h{};
    memcpy(h.magic, "FFECKPT1", 8);
    h.E = d.E;
    h.ndg = d.ndg;
    h.nfd = d.nfd;
    h.fd_cap = d.fd_slot ? d.fd_cap : 0;
    h.n_inst = c->n_inst;
    h.steps = c->steps;
    h.t = c->t;
    h.id_kind = c->id_kind;
    const std::vector<double>& prm = c->batch ? c->id_prm_inst : c->id_prm;
    h.id_nprm_total = (int64_t)prm.size();
    char* p = (char*)host_buf;
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(h.units, d.units, sizeof h.units, cudaMemcpyDeviceToHost));
    int fc = 0;
    if (d.fd_slot) CK(cudaMemcpy(&fc, &d.counts[5], sizeof(int), cudaMemcpyDeviceToHost));
    h.free_count = fc;
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    if (!prm.empty()) memcpy(p, prm.data(), prm.size() * sizeof(double));
    p += prm.size() * sizeof(double);
    CK(cudaMemcpy(p, c->un.p, NV * (size_t)(d.ndg + d.nfd) * sizeof(double), cudaMemcpyDeviceToHost));
    p += NV * (size_t)(d.ndg + d.nfd) * sizeof(double);
    CK(cudaMemcpy(p, d.mask, d.E, cudaMemcpyDeviceToHost));
    p += d.E;
    if (d.fd_slot) {
        CK(cudaMemcpy(p, d.fd_slot, sizeof(int) * d.E, cudaMemcpyDeviceToHost));
        p += sizeof(int) * d.E;
        CK(cudaMemcpy(p, d.slot_elem, sizeof(int) * d.fd_cap, cudaMemcpyDeviceToHost));
        p += sizeof(int) * d.fd_cap;
        CK(cudaMemcpy(p, d.free_slots, sizeof(int) * d.fd_cap, cudaMemcpyDeviceToHost));
    }
    *bytes = need;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_load(ffe_ctx* c, const void* host_buf, size_t bytes) try {
    g_err.clear();
    if (!c || !host_buf) return fail(FFE_EINVAL, "null argument");
    Dev& d = c->d;
    CkptHeader h;
    if (bytes < sizeof h) return fail(FFE_EINVAL, "checkpoint of %zu bytes is truncated", bytes);
    memcpy(&h, host_buf, sizeof h);
    if (memcmp(h.magic, "FFECKPT1", 8) != 0) return fail(FFE_EINVAL, "not a checkpoint of this library");
    if (h.E != d.E || h.ndg != d.ndg || h.nfd != d.nfd || h.fd_cap != (d.fd_slot ? d.fd_cap : 0) ||
        h.n_inst != c->n_inst)
        return fail(FFE_EINVAL, "checkpoint of a different mesh, order or FD pool");
    // sizes first (no allocation or arithmetic on an unchecked count), then every
    // index the kernels will follow; the context is changed only once all hold
    const size_t body = NV * (size_t)(d.ndg + d.nfd) * sizeof(double) + d.E +
                        (d.fd_slot ? sizeof(int) * ((size_t)d.E + 2 * (size_t)d.fd_cap) : 0);
    if (h.id_kind < FFE_ID_FAST_WAVE || h.id_kind > FFE_ID_BREAKDOWN_1D || h.id_nprm_total < 0 ||
        (size_t)h.id_nprm_total > (bytes - sizeof h) / sizeof(double) || h.steps < 0 || !std::isfinite(h.t) ||
        (c->batch && c->n_inst > 0 && h.id_nprm_total % c->n_inst != 0))
        return fail(FFE_EINVAL, "corrupt checkpoint header");
    const size_t need = sizeof h + (size_t)h.id_nprm_total * sizeof(double) + body;
    if (bytes < need) return fail(FFE_EINVAL, "checkpoint of %zu bytes, %zu expected", bytes, need);
    const char* p = (const char*)host_buf + sizeof h;
    std::vector<double> prm((size_t)h.id_nprm_total);
    if (!prm.empty()) memcpy(prm.data(), p, prm.size() * sizeof(double));
    p += prm.size() * sizeof(double);
    const char* state = p;
    p += NV * (size_t)(d.ndg + d.nfd) * sizeof(double);
    const unsigned char* mask = (const unsigned char*)p;
    p += d.E;
    for (int64_t e = 0; e < d.E; ++e)
        if (mask[e] > 1) return fail(FFE_EINVAL, "corrupt checkpoint: mask of element %lld is %d", (long long)e, mask[e]);
    std::vector<int> slot, selem, freel;
    if (d.fd_slot) {
        // the FD slot pool: an element is on FD exactly when it holds a slot,
        // slot <-> element both ways, and the free list holds the other slots once
        slot.resize(d.E);
        selem.resize(d.fd_cap);
        freel.resize(d.fd_cap);
        memcpy(slot.data(), p, sizeof(int) * d.E);
        memcpy(selem.data(), p + sizeof(int) * d.E, sizeof(int) * d.fd_cap);
        memcpy(freel.data(), p + sizeof(int) * ((size_t)d.E + d.fd_cap), sizeof(int) * d.fd_cap);
        int held = 0;
        for (int e = 0; e < d.E; ++e) {
            const int sl = slot[e];
            if (sl < -1 || sl >= d.fd_cap || (sl >= 0) != (mask[e] == 1) || (sl >= 0 && selem[sl] != e))
                return fail(FFE_EINVAL, "corrupt checkpoint: FD slot of element %d", e);
            held += sl >= 0;
        }
        for (int sl = 0; sl < d.fd_cap; ++sl) {
            const int e = selem[sl];
            if (e < -1 || e >= d.E || (e >= 0 && slot[e] != sl))
                return fail(FFE_EINVAL, "corrupt checkpoint: element of FD slot %d", sl);
        }
        if (h.free_count != d.fd_cap - held) return fail(FFE_EINVAL, "corrupt checkpoint: free FD slot count");
        std::vector<unsigned char> seen(d.fd_cap, 0);
        for (int64_t i = 0; i < h.free_count; ++i) {
            const int sl = freel[i];
            if (sl < 0 || sl >= d.fd_cap || selem[sl] != -1 || seen[sl])
                return fail(FFE_EINVAL, "corrupt checkpoint: free FD slot list");
            seen[sl] = 1;
        }
    }
    c->id_kind = (int)h.id_kind;
    if (c->batch) {
        c->id_prm_inst = prm;
        c->id_nprm = c->n_inst > 0 ? (int)(prm.size() / c->n_inst) : 0;
    } else {
        c->id_prm = prm;
    }
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(c->un.p, state, NV * (size_t)(d.ndg + d.nfd) * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.mask, mask, d.E, cudaMemcpyHostToDevice));
    if (d.fd_slot) {
        CK(cudaMemcpy(d.fd_slot, slot.data(), sizeof(int) * d.E, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d.slot_elem, selem.data(), sizeof(int) * d.fd_cap, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d.free_slots, freel.data(), sizeof(int) * d.fd_cap, cudaMemcpyHostToDevice));
        const int fc = (int)h.free_count;
        CK(cudaMemcpy(&d.counts[5], &fc, sizeof(int), cudaMemcpyHostToDevice));
        c->h_fd_slot = slot;
    }
    CK(cudaMemcpy(d.units, h.units, sizeof h.units, cudaMemcpyHostToDevice));
    c->t = h.t;
    c->steps = h.steps;
    return fill_dirichlet(c);
} catch (...) {
    return host_failure();
}

ffe_status ffe_constraints(ffe_ctx* c, const double* U_dev, double* out_host) try {
    g_err.clear();
    if (!c || !out_host) return fail(FFE_EINVAL, "null argument");
    const Dev& d = c->d;
    if (d.ks) return fail(FFE_ENOTIMPL, "constraint diagnostics are built for the flat metric");
    const int blocks = d.nsm * 4;
    ffe_status s;
    if (!c->d_cons && (s = dalloc(c, &c->d_cons, 4 * (size_t)blocks))) return s;
    double* part = c->d_cons;
    Field U{U_dev ? (double*)U_dev : c->un.p, NV, d.ndg, d.nfd};
    launch_constraints(d, U, part, blocks, c->st);
    std::vector<double> h(4 * (size_t)blocks);
    CK(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    out_host[0] = 0.0;
    out_host[1] = 1.0e308;
    out_host[2] = out_host[3] = 0.0;
    for (int b = 0; b < blocks; ++b) {
        out_host[0] = fmax(out_host[0], h[4 * b]);
        out_host[1] = fmin(out_host[1], h[4 * b + 1]);
        out_host[2] = fmax(out_host[2], h[4 * b + 2]);
        out_host[3] = fmax(out_host[3], h[4 * b + 3]);
    }
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_mask(ffe_ctx* c, const unsigned char** mask_dev, int* n_elem) try {
    g_err.clear();
    if (!c || !mask_dev) return fail(FFE_EINVAL, "null argument");
    *mask_dev = c->d.mask;
    if (n_elem) *n_elem = c->d.E;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_set_frozen_masks(ffe_ctx* c, int on) { return ffe_freeze_mask(c, on); }

ffe_status ffe_diagnostic(ffe_ctx* c, int kind, const double* args, double* out_host) try {
    g_err.clear();
    if (!c || !out_host) return fail(FFE_EINVAL, "null argument");
    const Dev& d = c->d;
    if (kind == FFE_DIAG_CONSTRAINTS) return ffe_constraints(c, nullptr, out_host);
    if (kind == FFE_DIAG_BFLUX_UPPER || kind == FFE_DIAG_LUMINOSITY) {
        if (!args) return fail(FFE_EINVAL, "surface diagnostics need args[0] = the radius");
        const double R = args[0];
        int inst, na;
        ffe_status s;
        if ((s = surface_target(c, args, R, &inst, &na))) return s;
        const bool upper = kind == FFE_DIAG_BFLUX_UPPER;
        if (upper && na % 2) return fail(FFE_EINVAL, "the equator lies on element boundaries only for even n_ang");
        const ffe_ctx::Surf* sf;
        if ((s = surface_get(c, R, upper, inst, &sf))) return s;
        return surface_sum(c, *sf, c->un.p, upper ? 1 : 0, nullptr, 0.0, out_host);
    }
    if (kind != FFE_DIAG_L2_ERR) return fail(FFE_EINVAL, "diagnostic kind %d", kind);
    int v0 = 3, nv = 3;
    if (args) {
        if (!(args[0] >= 0 && args[0] <= NV - 1 && args[1] >= 1 && args[0] + args[1] <= NV) ||
            args[0] != std::floor(args[0]) || args[1] != std::floor(args[1]))
            return fail(FFE_EINVAL, "L2 error: variables [%g, %g + %g) outside [0, 9)", args[0], args[0], args[1]);
        v0 = (int)args[0];
        nv = (int)args[1];
    }
    if (c->id_kind < 0) return fail(FFE_ESTATE, "L2 error: no initial data set");
    ffe_status s;
    if ((s = build_reference(c))) return s;
    const int blocks = d.nsm * 4;
    if (!c->d_cons && (s = dalloc(c, &c->d_cons, 4 * (size_t)blocks))) return s;
    Field R{c->d_ref, NV, d.ndg, d.nfd};
    launch_l2_err(d, c->un, R, v0, nv, c->d_cons, blocks, c->st);
    std::vector<double> h(blocks);
    CK(cudaMemcpyAsync(h.data(), c->d_cons, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double sum = 0.0;
    for (double x : h) sum += x;
    int64_t npts = 0;
    for (int e = 0; e < d.E; ++e) {
        const int P = host_P(c, e);
        npts += c->ref_mask[e] ? (int64_t)(2 * P + 1) * (2 * P + 1) * (2 * P + 1) : (int64_t)(P + 1) * (P + 1) * (P + 1);
    }
    out_host[0] = std::sqrt(sum / (double)npts);
    out_host[1] = (double)npts;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_coords(ffe_ctx* c, double* xyz_dg_dev, double* xyz_fd_dev) try {
    g_err.clear();
    if (!c) return fail(FFE_EINVAL, "null context");
    const Dev& d = c->d;
    if (xyz_fd_dev && (!d.xyz_fd || d.fd_slot))
        return fail(FFE_ENOTIMPL, "FD centres in state-vector order need one FD slot per element (no FD slot pool)");
    if (xyz_dg_dev)
        CK(cudaMemcpyAsync(xyz_dg_dev, d.xyz_dg, 3 * (size_t)d.ndg * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    if (xyz_fd_dev)
        CK(cudaMemcpyAsync(xyz_fd_dev, d.xyz_fd, 3 * (size_t)d.nfd * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_eval_recip(const double* x_dev, double* y_dev, int64_t n, void* cuda_stream) try {
    g_err.clear();
    if (n < 0 || (n > 0 && (!x_dev || !y_dev))) return fail(FFE_EINVAL, "bad argument");
    if (n == 0) return FFE_OK;
    launch_eval_recip(x_dev, y_dev, n, (cudaStream_t)cuda_stream);
    CK(cudaGetLastError());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_fp64_fma_rate(void* cuda_stream, double* tflops_host) try {
    g_err.clear();
    if (!tflops_host) return fail(FFE_EINVAL, "null argument");
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    float ms = 0.0f;
    const double flops = launch_fma_probe(nsm, 1 << 16, (cudaStream_t)cuda_stream, &ms);
    CK(cudaGetLastError());
    if (!(ms > 0.0f)) return fail(FFE_ECUDA, "the probe's events gave no duration");
    *tflops_host = flops / (ms * 1e-3) / 1e12;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

const char* ffe_last_error(void) { return g_err.c_str(); }

namespace {
// Every node and FD cell index of a context fits a 32-bit int: at most
// INT_MAX / (2 Pmax + 1)^3 elements (1.6 M at P = 5, beyond what fits in HBM).
ffe_status check_count(int64_t E, int Pmax, const char* who) {
    const int64_t per = (int64_t)(2 * Pmax + 1) * (2 * Pmax + 1) * (2 * Pmax + 1);
    if (E < 1 || E > INT32_MAX / per)
        return fail(FFE_EINVAL, "%s: %lld elements (1 to %lld at P = %d)", who, (long long)E, (long long)(INT32_MAX / per), Pmax);
    return FFE_OK;
}

// Scheme parameters: finite, damping and filter strengths non-negative, a
// positive step or CFL data, indicator and WENO constants positive where used,
// known constraint mode and reconstruction.
ffe_status check_scheme(const ffe_params& p, const char* who) {
    const double v[] = {p.eta, p.kappa_psi, p.kappa_phi, p.cfl, p.c_over_D, p.dt, p.filter_a, p.filter_b,
                        p.tci_alpha, p.weno_eps, p.omega_star};
    for (double x : v)
        if (!std::isfinite(x)) return fail(FFE_EINVAL, "%s: a scheme parameter is not finite", who);
    if (p.eta < 0 || p.kappa_psi < 0 || p.kappa_phi < 0) return fail(FFE_EINVAL, "%s: negative damping", who);
    if (p.dt < 0 || (p.dt == 0 && !(p.cfl > 0 && p.c_over_D > 0)))
        return fail(FFE_EINVAL, "%s: need dt > 0 or cfl > 0 and c_over_D > 0", who);
    if (p.filter_on && (p.filter_a < 0 || !(p.filter_b > 0)))
        return fail(FFE_EINVAL, "%s: filter needs a >= 0 and b > 0", who);
    if (p.constraint_mode < FFE_RELAX || p.constraint_mode > FFE_RELAX_THEN_HARD)
        return fail(FFE_EINVAL, "%s: constraint mode %d", who, p.constraint_mode);
    if (p.recon != FFE_RECON_WENO5Z && p.recon != FFE_RECON_MP5) return fail(FFE_EINVAL, "%s: reconstruction %d", who, p.recon);
    if (p.fd_chunk < 0) return fail(FFE_EINVAL, "%s: fd_chunk %d < 0", who, p.fd_chunk);
    if (p.fd_capacity < 0) return fail(FFE_EINVAL, "%s: fd_capacity %d < 0", who, p.fd_capacity);
    if (p.tci_on && !(p.tci_alpha > 0)) return fail(FFE_EINVAL, "%s: indicator needs alpha > 0", who);
    if (p.tci_on && p.recon == FFE_RECON_WENO5Z && !(p.weno_eps > 0))
        return fail(FFE_EINVAL, "%s: WENO5-Z needs eps > 0", who);
    return FFE_OK;
}
// Streaming multiprocessors of the current device: launch shapes (persistent
// grids, grid-stride loops) are multiples of it.
ffe_status query_sms(ffe_ctx* c) {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    c->d.nsm = nsm > 0 ? nsm : 1;
    return FFE_OK;
}
}  // namespace

ffe_status ffe_create(const ffe_domain* domain, const ffe_elements* elements, int P, const ffe_metric* metric,
                      const ffe_params* params, void* cuda_stream, ffe_ctx** out) try {
    g_err.clear();
    if (!domain || !elements || !metric || !params || !out) return fail(FFE_EINVAL, "null argument");
    *out = nullptr;
    if (P < 2 || P > 6) return fail(FFE_EINVAL, "order P=%d outside [2, 6]", P);
    if (params->tci_on && P < 3) return fail(FFE_EINVAL, "FD subcells need P >= 3 (6-point projection stencil)");
    if (domain->kind != FFE_DOMAIN_BOX && domain->kind != FFE_DOMAIN_SHELL6)
        return fail(FFE_EINVAL, "domain kind %d", domain->kind);
    if (metric->kind != FFE_METRIC_MINKOWSKI && metric->kind != FFE_METRIC_KERR_SCHILD)
        return fail(FFE_EINVAL, "metric kind %d", metric->kind);
    if (metric->kind == FFE_METRIC_KERR_SCHILD) {
        if (domain->kind != FFE_DOMAIN_SHELL6) return fail(FFE_EINVAL, "Kerr-Schild needs a shell domain");
        if (params->tci_on && params->fd_corrector)
            return fail(FFE_ENOTIMPL, "the FD flux corrector is defined for Cartesian meshes, not the Kerr-Schild background");
        if (params->tci_on && (domain->bc_lo[0] != FFE_BC_DIRICHLET || domain->bc_hi[0] != FFE_BC_DIRICHLET))
            return fail(FFE_ENOTIMPL, "FD subcells on the Kerr-Schild background take Dirichlet shell boundaries");
        if (!(metric->M > 0) || !(fabs(metric->a) < 1)) return fail(FFE_EINVAL, "need M > 0 and |a| < 1");
        if (P < 3 || P > 5) return fail(FFE_EINVAL, "curved elements support 3 <= P <= 5");
    }
    if (domain->shell_ks != 0) {
        if (domain->shell_ks != 1) return fail(FFE_EINVAL, "shell_ks = %d (0 or 1)", domain->shell_ks);
        if (domain->kind != FFE_DOMAIN_SHELL6 || metric->kind != FFE_METRIC_KERR_SCHILD)
            return fail(FFE_EINVAL, "shell_ks needs a shell on the Kerr-Schild metric");
        if (params->tci_on)
            return fail(FFE_ENOTIMPL, "FD subcells are not built for the spherical Kerr-Schild shell (tci_on = 0)");
    }
    if (domain->kind == FFE_DOMAIN_SHELL6) {
        if (!(domain->r_in > 0) || !(domain->r_out > domain->r_in)) return fail(FFE_EINVAL, "need 0 < r_in < r_out");
        if (elements->n[0] < 1 || elements->n[2] < 1) return fail(FFE_EINVAL, "shell needs n[0], n[2] >= 1");
        if (P < 3 || P > 5) return fail(FFE_EINVAL, "curved elements support 3 <= P <= 5");
        for (int k : {domain->bc_lo[0], domain->bc_hi[0]})
            if (k < FFE_BC_DIRICHLET || k > FFE_BC_OUTFLOW) return fail(FFE_EINVAL, "shell boundary kind %d", k);
    }
    for (int dd = 0; dd < 3 && domain->kind == FFE_DOMAIN_BOX; ++dd) {
        if (elements->n[dd] < 1) return fail(FFE_EINVAL, "elements n[%d] = %d", dd, elements->n[dd]);
        if (!(domain->hi[dd] > domain->lo[dd])) return fail(FFE_EINVAL, "empty box along axis %d", dd);
        for (int k : {domain->bc_lo[dd], domain->bc_hi[dd]})
            if (k < FFE_BC_PERIODIC || k > FFE_BC_OUTFLOW) return fail(FFE_EINVAL, "boundary kind %d", k);
        if ((domain->bc_lo[dd] == FFE_BC_PERIODIC) != (domain->bc_hi[dd] == FFE_BC_PERIODIC))
            return fail(FFE_EINVAL, "periodic axis %d needs periodic at both ends", dd);
    }
    if (params->tci_on && (params->tci_M < 1 || params->tci_M > P)) return fail(FFE_EINVAL, "tci_M=%d", params->tci_M);
    ffe_status st0;
    if ((st0 = check_scheme(*params, "parameters"))) return st0;
    if (domain->kind == FFE_DOMAIN_SHELL6) {
        if (!std::isfinite(domain->r_out)) return fail(FFE_EINVAL, "need a finite r_out");
        st0 = check_count(6 * (int64_t)elements->n[0] * elements->n[0] * elements->n[2], P, "shell");
    } else {
        for (int dd = 0; dd < 3; ++dd)
            if (!std::isfinite(domain->lo[dd]) || !std::isfinite(domain->hi[dd]))
                return fail(FFE_EINVAL, "box bounds along axis %d are not finite", dd);
        st0 = check_count((int64_t)elements->n[0] * elements->n[1] * elements->n[2], P, "box");
    }
    if (st0) return st0;
    if (metric->kind == FFE_METRIC_KERR_SCHILD && !std::isfinite(metric->M)) return fail(FFE_EINVAL, "need a finite M");

    ffe_ctx* c = new ffe_ctx();
    if (ffe_status sq = query_sms(c)) {
        delete c;
        return sq;
    }
    c->dom = *domain;
    c->el = *elements;
    c->met = *metric;
    c->prm = *params;
    c->st = (cudaStream_t)cuda_stream;
    Dev& d = c->d;
    if (domain->kind == FFE_DOMAIN_SHELL6) {
        c->shell.r_in = domain->r_in;
        c->shell.c = 0.5 * log(domain->r_out / domain->r_in);
        c->shell.na = elements->n[0];
        c->shell.nr = elements->n[2];
        c->shell.a = domain->shell_ks ? metric->a : 0.0;
        d.E = 6 * elements->n[0] * elements->n[0] * elements->n[2];
    } else {
        c->nx = elements->n[0];
        c->ny = elements->n[1];
        c->nz = elements->n[2];
        for (int dd = 0; dd < 3; ++dd) c->h[dd] = (domain->hi[dd] - domain->lo[dd]) / elements->n[dd];
        d.E = c->nx * c->ny * c->nz;
    }
    d.P = P;
    d.np1 = P + 1;
    d.nn = d.np1 * d.np1 * d.np1;
    d.nc = 2 * P + 1;
    d.ncell = d.nc * d.nc * d.nc;
    d.ndg = (int64_t)d.E * d.nn;
    d.nfd = (int64_t)d.E * d.ncell;
    d.eta = params->constraint_mode == FFE_HARD ? 0.0 : params->eta;
    d.kpsi = params->kappa_psi;
    d.kphi = params->kappa_phi;
    d.weno_eps = params->weno_eps;
    d.recon = params->recon;
    d.omega = params->omega_star;
    d.mode = params->constraint_mode;
    d.filter_on = params->filter_on;
    d.tci_on = params->tci_on;
    c->tci_param = params->tci_on;
    d.fd_corr = params->fd_corrector;
    ffe_status s;
    auto bail = [&](ffe_status s) { ffe_destroy(c); return s; };
    build_tables(P, params->filter_a, params->filter_b, params->tci_M, c->tabs_h[P]);
    c->tab = c->tabs_h[P];
    if ((s = (domain->kind == FFE_DOMAIN_SHELL6 ? build_shell(c) : build_box(c)))) return bail(s);
    d.dt = params->dt > 0 ? params->dt : params->cfl * c->dxmin / c->lam_max * params->c_over_D;
    const int cap = params->fd_capacity > 0 && params->fd_capacity < d.E ? params->fd_capacity : d.E;
    if ((s = finish_create(c, cap, {P}))) return bail(s);
    *out = c;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_create_batch(int n_inst, const ffe_domain* doms, const ffe_elements* els, const int* Ps,
                            const ffe_metric* metric, const ffe_params* params, int fd_capacity, void* cuda_stream,
                            ffe_ctx** out) try {
    g_err.clear();
    if (n_inst < 1 || !doms || !els || !Ps || !metric || !params || !out) return fail(FFE_EINVAL, "bad argument");
    *out = nullptr;
    if (metric->kind != FFE_METRIC_MINKOWSKI) return fail(FFE_ENOTIMPL, "batched contexts are flat-space shells");
    if (fd_capacity < 0) return fail(FFE_EINVAL, "fd_capacity < 0");
    const ffe_params& p0 = params[0];
    int64_t n_all = 0;
    for (int i = 0; i < n_inst; ++i) {
        const ffe_domain& dm = doms[i];
        const ffe_params& pi = params[i];
        char who[32];
        snprintf(who, sizeof who, "instance %d", i);
        ffe_status st0;
        if ((st0 = check_scheme(pi, who))) return st0;
        if (dm.kind != FFE_DOMAIN_SHELL6) return fail(FFE_EINVAL, "instance %d: batched instances are shells", i);
        if (dm.shell_ks) return fail(FFE_EINVAL, "instance %d: shell_ks needs the Kerr-Schild metric", i);
        if (!(dm.r_in > 0) || !(dm.r_out > dm.r_in)) return fail(FFE_EINVAL, "instance %d: need 0 < r_in < r_out", i);
        if (els[i].n[0] < 1 || els[i].n[2] < 1) return fail(FFE_EINVAL, "instance %d: element counts", i);
        if (Ps[i] < 3 || Ps[i] > 5) return fail(FFE_EINVAL, "instance %d: order %d outside [3, 5]", i, Ps[i]);
        for (int k : {dm.bc_lo[0], dm.bc_hi[0]})
            if (k < FFE_BC_DIRICHLET || k > FFE_BC_OUTFLOW) return fail(FFE_EINVAL, "instance %d: boundary kind %d", i, k);
        if (pi.eta != p0.eta || pi.kappa_psi != p0.kappa_psi || pi.kappa_phi != p0.kappa_phi ||
            pi.filter_on != p0.filter_on || pi.filter_a != p0.filter_a || pi.filter_b != p0.filter_b ||
            pi.tci_on != p0.tci_on || pi.tci_M != p0.tci_M || pi.tci_alpha != p0.tci_alpha ||
            pi.weno_eps != p0.weno_eps || pi.fd_corrector != p0.fd_corrector || pi.recon != p0.recon ||
            pi.constraint_mode != p0.constraint_mode || pi.fd_chunk != p0.fd_chunk)
            return fail(FFE_EINVAL, "instance %d: scheme parameters differ from instance 0", i);
        if (!std::isfinite(dm.r_out)) return fail(FFE_EINVAL, "instance %d: need a finite r_out", i);
        if (p0.tci_on && (p0.tci_M < 1 || p0.tci_M > Ps[i])) return fail(FFE_EINVAL, "tci_M=%d", p0.tci_M);
        n_all += 6 * (int64_t)els[i].n[0] * els[i].n[0] * els[i].n[2];
        if ((st0 = check_count(n_all, 5, "batch"))) return st0;
    }
    ffe_ctx* c = new ffe_ctx();
    if (ffe_status sq = query_sms(c)) {
        delete c;
        return sq;
    }
    auto bail = [&](ffe_status s) { ffe_destroy(c); return s; };
    c->batch = true;
    c->n_inst = n_inst;
    c->dom = doms[0];
    c->el = els[0];
    c->met = *metric;
    c->prm = p0;
    c->st = (cudaStream_t)cuda_stream;
    c->doms.assign(doms, doms + n_inst);
    Dev& d = c->d;
    int Pmax = 0, E = 0;
    std::vector<int> orders;
    for (int i = 0; i < n_inst; ++i) {
        InstInfo in{};
        in.r_in = doms[i].r_in;
        in.c = 0.5 * log(doms[i].r_out / doms[i].r_in);
        in.omega = params[i].omega_star;
        in.na = els[i].n[0];
        in.nr = els[i].n[2];
        in.e0 = E;
        in.P = Ps[i];
        c->insts.push_back(in);
        const int Ei = 6 * in.na * in.na * in.nr;
        for (int k = 0; k < Ei; ++k) { c->h_eP.push_back(Ps[i]); c->h_einst.push_back(i); }
        E += Ei;
        Pmax = Ps[i] > Pmax ? Ps[i] : Pmax;
        bool seen = false;
        for (int q : orders) seen |= q == Ps[i];
        if (!seen) orders.push_back(Ps[i]);
    }
    d.E = E;
    d.P = Pmax;
    d.np1 = Pmax + 1;
    d.nn = d.np1 * d.np1 * d.np1;
    d.nc = 2 * Pmax + 1;
    d.ncell = d.nc * d.nc * d.nc;
    d.ndg = (int64_t)E * d.nn;
    d.eta = p0.constraint_mode == FFE_HARD ? 0.0 : p0.eta;
    d.kpsi = p0.kappa_psi;
    d.kphi = p0.kappa_phi;
    d.weno_eps = p0.weno_eps;
    d.recon = p0.recon;
    d.omega = p0.omega_star;
    d.mode = p0.constraint_mode;
    d.filter_on = p0.filter_on;
    d.tci_on = p0.tci_on;
    c->tci_param = p0.tci_on;
    d.fd_corr = p0.fd_corrector;
    d.curved = 1;
    for (int P : orders) build_tables(P, p0.filter_a, p0.filter_b, p0.tci_M, c->tabs_h[P]);
    // geometry of every instance into the element slots
    const int64_t ndg = d.ndg;
    std::vector<double> xdg(3 * (size_t)ndg, 0.0), geo(9 * (size_t)ndg, 0.0);
    std::vector<int> nbr(6 * E, -1), nbf(6 * E, -1), orient(6 * E, 0), bc(6 * E, 0), bface(6 * E, -1);
    int nbfd = 0;
    for (int i = 0; i < n_inst; ++i) {
        InstInfo& in = c->insts[i];
        const ShellGeo g{in.r_in, in.c, in.na, in.nr};
        const int P = in.P, np1 = P + 1, nn = np1 * np1 * np1, Ei = 6 * in.na * in.na * in.nr;
        const Tables& T = c->tabs_h[P];
        MapFn map = [g](int e, const double xi[3], double x[3], double ij[3][3]) { shell_map(g, e, xi, x, ij); };
        double dmin = 1e300;
        for (int el = 0; el < Ei; ++el) {
            const int e = in.e0 + el;
            for (int q = 0; q < nn; ++q) {
                const int ci[3] = {q % np1, (q / np1) % np1, q / (np1 * np1)};
                const double xi[3] = {T.x[ci[0]], T.x[ci[1]], T.x[ci[2]]};
                double x[3], ij[3][3];
                map(el, xi, x, ij);
                const int64_t p = (int64_t)e * d.nn + q;
                for (int a = 0; a < 3; ++a) xdg[a * ndg + p] = x[a];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) geo[(3 * a + b) * ndg + p] = ij[a][b];
            }
            for (int q = 0; q < nn; ++q) {
                const int ci[3] = {q % np1, (q / np1) % np1, q / (np1 * np1)};
                for (int a = 0; a < 3; ++a) {
                    if (ci[a] == P) continue;
                    const int q2 = q + (a == 0 ? 1 : (a == 1 ? np1 : np1 * np1));
                    double s2 = 0.0;
                    for (int b = 0; b < 3; ++b) {
                        const double dx = xdg[b * ndg + (int64_t)e * d.nn + q2] - xdg[b * ndg + (int64_t)e * d.nn + q];
                        s2 += dx * dx;
                    }
                    dmin = fmin(dmin, sqrt(s2));
                }
            }
        }
        in.dt = params[i].dt > 0 ? params[i].dt : params[i].cfl * dmin * params[i].c_over_D;
        std::vector<double> xn(T.x, T.x + np1);
        std::vector<int> lnbr, lnbf, lor;
        match_faces(Ei, map, xn, np1, doms[i].r_out, lnbr, lnbf, lor);
        for (int el = 0; el < Ei; ++el)
            for (int f = 0; f < 6; ++f) {
                const int e = in.e0 + el, k = 6 * el + f;
                if (lnbr[k] == -2) return bail(fail(FFE_EINVAL, "instance %d: no orientation for a face", i));
                if (lnbr[k] >= 0) {
                    nbr[6 * e + f] = lnbr[k] + in.e0;
                    nbf[6 * e + f] = lnbf[k];
                    orient[6 * e + f] = lor[k];
                    continue;
                }
                const int ir = (el / (in.na * in.na)) % in.nr;
                int kind;
                if (f == 4 && ir == 0) kind = doms[i].bc_lo[0];
                else if (f == 5 && ir == in.nr - 1) kind = doms[i].bc_hi[0];
                else return bail(fail(FFE_EINVAL, "instance %d: unmatched interior face", i));
                bc[6 * e + f] = kind;
                if (kind == FFE_BC_DIRICHLET) bface[6 * e + f] = nbfd++;
            }
    }
    c->nbf = nbfd;
    c->h_bface = bface;
    if (ffe_status sg = set_ginterp(c, nbr)) return bail(sg);
    d.dt = c->insts[0].dt;
    ffe_status s;
    double *d_xdg, *d_geo, *d_bdg, *d_bfd, *d_ijac;
    int *d_nbr, *d_nbf, *d_bc, *d_bface, *d_or;
    if ((s = dalloc(c, &d_xdg, xdg.size()))) return bail(s);
    if ((s = dalloc(c, &d_geo, geo.size()))) return bail(s);
    if ((s = dalloc(c, &d_ijac, 3 * (size_t)E))) return bail(s);
    if ((s = dalloc(c, &d_nbr, nbr.size()))) return bail(s);
    if ((s = dalloc(c, &d_nbf, nbf.size()))) return bail(s);
    if ((s = dalloc(c, &d_or, orient.size()))) return bail(s);
    if ((s = dalloc(c, &d_bc, bc.size()))) return bail(s);
    if ((s = dalloc(c, &d_bface, bface.size()))) return bail(s);
    if ((s = dalloc(c, &d_bdg, (size_t)(nbfd > 0 ? nbfd : 1) * NV * d.np1 * d.np1))) return bail(s);
    if ((s = dalloc(c, &d_bfd, (size_t)(nbfd > 0 ? nbfd : 1) * NV * GH * d.nc * d.nc))) return bail(s);
    if (cudaMemcpy(d_xdg, xdg.data(), xdg.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_nbf, nbf.data(), nbf.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_or, orient.data(), orient.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_bc, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(d_bface, bface.data(), bface.size() * 4, cudaMemcpyHostToDevice))
        return bail(fail(FFE_ECUDA, "geometry upload"));
    d.xyz_dg = d_xdg;
    d.xyz_fd = nullptr;
    d.geo = d_geo;
    d.ijac = d_ijac;
    d.nbr = d_nbr;
    d.nbr_face = d_nbf;
    d.orient = d_or;
    d.bc = d_bc;
    d.bface = d_bface;
    d.bdg = d_bdg;
    d.bfd = d_bfd;
    const int cap = fd_capacity > 0 && fd_capacity < E ? fd_capacity : E;
    if ((s = finish_create(c, cap, orders))) return bail(s);
    *out = c;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_layout(ffe_ctx* c, int* elem_P, int* fd_slot, int* elem_inst, int* inst_first, int* n_inst) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    const Dev& d = c->d;
    CK(cudaStreamSynchronize(c->st));
    for (int e = 0; e < d.E; ++e) {
        if (elem_P) elem_P[e] = host_P(c, e);
        if (elem_inst) elem_inst[e] = c->batch ? c->h_einst[e] : 0;
    }
    if (fd_slot) {
        if (d.fd_slot) CK(cudaMemcpy(fd_slot, d.fd_slot, d.E * sizeof(int), cudaMemcpyDeviceToHost));
        else
            for (int e = 0; e < d.E; ++e) fd_slot[e] = e;
    }
    if (inst_first) {
        for (int i = 0; i < c->n_inst; ++i) inst_first[i] = c->batch ? c->insts[i].e0 : 0;
        inst_first[c->n_inst] = d.E;
    }
    if (n_inst) *n_inst = c->n_inst;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_set_initial_batch(ffe_ctx* c, int id_kind, const double* id_params, int n_params, int flags) try {
    g_err.clear();
    if (!c) return fail(FFE_EINVAL, "null context");
    if (id_kind < FFE_ID_FAST_WAVE || id_kind > FFE_ID_DIPOLE) return fail(FFE_EINVAL, "initial data kind %d", id_kind);
    if (n_params < 0 || (n_params > 0 && !id_params)) return fail(FFE_EINVAL, "bad initial-data parameters");
    if (flags & FFE_INIT_VIA_FD) return fail(FFE_ENOTIMPL, "an FD start is not built for batches (FD slot pool)");
    c->id_kind = id_kind;
    if (c->batch) {
        c->id_nprm = n_params;
        c->id_prm_inst.assign(id_params, id_params + (size_t)n_params * c->n_inst);
    } else {
        c->id_prm.assign(id_params, id_params + n_params);
    }
    return set_initial_impl(c, id_kind, (flags & FFE_INIT_KEEP_MASK) != 0, (flags & FFE_INIT_VIA_FD) != 0);
} catch (...) {
    return host_failure();
}

ffe_status ffe_set_initial(ffe_ctx* c, int id_kind, const double* id_params, int n_params, int flags) try {
    g_err.clear();
    if (!c) return fail(FFE_EINVAL, "null context");
    if (id_kind < FFE_ID_FAST_WAVE || id_kind > FFE_ID_BREAKDOWN_1D) return fail(FFE_EINVAL, "initial data kind %d", id_kind);
    if (n_params < 0 || (n_params > 0 && !id_params)) return fail(FFE_EINVAL, "bad initial-data parameters");
    if ((flags & FFE_INIT_VIA_FD) && (flags & FFE_INIT_KEEP_MASK))
        return fail(FFE_EINVAL, "FFE_INIT_VIA_FD and FFE_INIT_KEEP_MASK exclude each other");
    if ((flags & FFE_INIT_VIA_FD) && (c->d.ks || !c->d.tci_on))
        return fail(FFE_EINVAL, "an FD start needs the indicator on and a flat metric");
    c->id_kind = id_kind;
    c->id_prm.assign(id_params, id_params + n_params);
    if (c->batch) {
        c->id_nprm = n_params;
        c->id_prm_inst.clear();
        for (int i = 0; i < c->n_inst; ++i) c->id_prm_inst.insert(c->id_prm_inst.end(), id_params, id_params + n_params);
    }
    return set_initial_impl(c, id_kind, (flags & FFE_INIT_KEEP_MASK) != 0, (flags & FFE_INIT_VIA_FD) != 0);
} catch (...) {
    return host_failure();
}

ffe_status ffe_rhs(ffe_ctx* c, const double* U_dev, double* dUdt_dev) try {
    g_err.clear();
    if (!c || !U_dev || !dUdt_dev) return fail(FFE_EINVAL, "null argument");
    if (c->id_kind < 0) return fail(FFE_ESTATE, "no initial data set (boundary data undefined)");
    const Dev& d = c->d;
    Field U{(double*)U_dev, NV, d.ndg, d.nfd}, R{dUdt_dev, NV, d.ndg, d.nfd};
    launch_build_lists(d, c->st);
    launch_current(d, U, c->J, nullptr, 0, c->st);
    if (d.curved)
        launch_dg_substep_curved(d, SUB_RHS, U, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, R, R, c->G1,
                                 c->st);
    else
        launch_dg_substep(d, SUB_RHS, U, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, R, R, c->G1, c->st);
    launch_fd_substep(d, SUB_RHS, d.fd_list, 1, U, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, R, R,
                      c->G1, c->st);
    CK(cudaGetLastError());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_step(ffe_ctx* c, int nsteps) try {
    g_err.clear();
    if (!c || nsteps < 0) return fail(FFE_EINVAL, "bad argument");
    if (c->id_kind < 0) return fail(FFE_ESTATE, "no initial data set");
    return run_steps(c, nsteps);
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_state(ffe_ctx* c, double** U_dev, unsigned char** mask_dev) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    if (U_dev) *U_dev = c->un.p;
    if (mask_dev) *mask_dev = c->d.mask;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

namespace {
// A caller's mask (host copy) before it replaces the context's: bytes 0 (DG)
// or 1 (FD) only, and in an FD slot pool exactly the elements that hold a slot
// on FD (elements change pool slots only through the indicator's switches).
ffe_status check_mask(ffe_ctx* c, const unsigned char* m) {
    const Dev& d = c->d;
    for (int e = 0; e < d.E; ++e) {
        if (m[e] > 1) return fail(FFE_EINVAL, "mask of element %d is %d (0 = DG, 1 = FD)", e, m[e]);
        if (m[e] == 1 && d.ks && !d.metfd)
            return fail(FFE_ENOTIMPL, "FD elements on the Kerr-Schild background need a context created with the "
                                      "indicator on (the metric at the FD points is tabulated then)");
    }
    if (d.fd_slot) {
        std::vector<int> slot(d.E);
        CK(cudaMemcpyAsync(slot.data(), d.fd_slot, sizeof(int) * d.E, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int e = 0; e < d.E; ++e)
            if ((slot[e] >= 0) != (m[e] == 1))
                return fail(FFE_EINVAL, "mask of element %d does not match the FD slot pool", e);
    }
    return FFE_OK;
}
}  // namespace

ffe_status ffe_set_state(ffe_ctx* c, const double* U_dev, const unsigned char* mask_dev) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    const Dev& d = c->d;
    if (mask_dev) {
        std::vector<unsigned char> m(d.E);
        CK(cudaMemcpyAsync(m.data(), mask_dev, d.E, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        ffe_status s;
        if ((s = check_mask(c, m.data()))) return s;
    }
    if (U_dev) CK(cudaMemcpyAsync(c->un.p, U_dev, NV * (d.ndg + d.nfd) * 8, cudaMemcpyDeviceToDevice, c->st));
    if (mask_dev) CK(cudaMemcpyAsync(d.mask, mask_dev, d.E, cudaMemcpyDeviceToDevice, c->st));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_download(ffe_ctx* c, double* U_host, unsigned char* mask_host) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    const Dev& d = c->d;
    if (U_host) CK(cudaMemcpyAsync(U_host, c->un.p, NV * (d.ndg + d.nfd) * 8, cudaMemcpyDeviceToHost, c->st));
    if (mask_host) CK(cudaMemcpyAsync(mask_host, d.mask, d.E, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_upload(ffe_ctx* c, const double* U_host, const unsigned char* mask_host) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    const Dev& d = c->d;
    ffe_status s;
    if (mask_host && (s = check_mask(c, mask_host))) return s;
    if (U_host) CK(cudaMemcpyAsync(c->un.p, U_host, NV * (d.ndg + d.nfd) * 8, cudaMemcpyHostToDevice, c->st));
    if (mask_host) CK(cudaMemcpyAsync(d.mask, mask_host, d.E, cudaMemcpyHostToDevice, c->st));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_info(ffe_ctx* c, ffe_info* info) try {
    if (!c || !info) return fail(FFE_EINVAL, "null argument");
    const Dev& d = c->d;
    info->n_elem = d.E;
    info->P = d.P;
    info->np1 = d.np1;
    info->nc = d.nc;
    info->n_dg = d.ndg;
    info->n_fd = d.nfd;
    info->n_state = NV * (d.ndg + d.nfd);
    info->dt = d.dt;
    info->dxmin = c->dxmin;
    info->t = c->t;
    info->steps = c->steps;
    std::vector<unsigned char> m(d.E);
    CK(cudaMemcpyAsync(m.data(), d.mask, d.E, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    int n = 0;
    for (unsigned char x : m) n += x;
    info->n_fd_elem = n;
    unsigned long long u[3] = {0, 0, 0};
    CK(cudaMemcpy(u, d.units, sizeof u, cudaMemcpyDeviceToHost));
    info->node_updates = (int64_t)u[0];
    info->fd_elem_updates = (int64_t)u[1];
    info->dg_elem_updates = (int64_t)u[2];
    info->dg_ctas_per_sm[0] = d.dg_grid / d.nsm;
    info->dg_ctas_per_sm[1] = d.dg_grid_lo / d.nsm;
    info->dg_ctas_per_sm[2] = d.dg_grid_lo2 / d.nsm;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_get_status(ffe_ctx* c, int* bits) try {
    if (!c || !bits) return fail(FFE_EINVAL, "null argument");
    CK(cudaMemcpyAsync(bits, c->d.counts + 4, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemsetAsync(c->d.counts + 4, 0, sizeof(int), c->st));
    CK(cudaStreamSynchronize(c->st));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_tci_ratio(ffe_ctx* c, const double* U_dev, double* ratio_dev) try {
    if (!c || !U_dev || !ratio_dev) return fail(FFE_EINVAL, "null argument");
    launch_tci_ratio(c->d, U_dev, ratio_dev, c->st);
    CK(cudaGetLastError());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_near_threshold(ffe_ctx* c, int* idx, int cap, int* n) try {
    if (!c || !n || (cap > 0 && !idx)) return fail(FFE_EINVAL, "bad argument");
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, c->d.counts + 3, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    cnt = cnt > 4096 ? 4096 : cnt;
    *n = cnt;
    if (cap > 0 && cnt > 0)
        CK(cudaMemcpy(idx, c->d.near_list, (size_t)(cnt < cap ? cnt : cap) * sizeof(int), cudaMemcpyDeviceToHost));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_launch_count(ffe_ctx* c, int64_t* n) try {
    if (!c || !n) return fail(FFE_EINVAL, "null argument");
    *n = g_launch_counter;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_freeze_mask(ffe_ctx* c, int on) try {
    g_err.clear();
    if (!c) return fail(FFE_EINVAL, "null context");
    CK(cudaStreamSynchronize(c->st));
    const int want = on ? 0 : c->tci_param;
    if (c->d.tci_on != want) {
        c->d.tci_on = want;
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
    }
    return FFE_OK;
} catch (...) {
    return host_failure();
}

static ffe_status adjoint_ready(ffe_ctx* c) {
    const Dev& d = c->d;
    if (!d.curved || d.ks || c->batch) return fail(FFE_ENOTIMPL, "the adjoint is built for flat-metric shells");
    if (c->dom.bc_lo[0] == FFE_BC_OUTFLOW || c->dom.bc_hi[0] == FFE_BC_OUTFLOW)
        return fail(FFE_ENOTIMPL, "the adjoint is not built for outflow boundaries");
    if (d.recon != FFE_RECON_WENO5Z) return fail(FFE_ENOTIMPL, "the adjoint is built for WENO5-Z reconstruction");
    if (d.tci_on) return fail(FFE_ESTATE, "the adjoint differentiates a fixed mask: freeze it first (ffe_freeze_mask)");
    std::vector<unsigned char> m(d.E);
    CK(cudaMemcpyAsync(m.data(), d.mask, d.E, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->adj_fd = false;
    for (unsigned char x : m) c->adj_fd |= x != 0;
    if (c->adj_ready) return FFE_OK;
    AdjArgs& a = c->adj;
    ffe_status s;
    for (Field* f : {&a.U2, &a.R3, &a.R4, &a.T3, &a.T4, &a.U3, &a.U4, &a.F2, &a.F3, &a.F4, &a.W, &a.lam, &a.ubar,
                     &a.F2b, &a.F3b, &a.F4b, &a.tmp, &a.tmp2})
        if ((s = alloc_field(c, *f, NV))) return s;
    for (Field* f : {&a.G1, &a.G2, &a.G3, &a.G4, &a.G1b, &a.G2b, &a.G3b, &a.G4b})
        if ((s = alloc_field(c, *f, NG))) return s;
    if ((s = dalloc(c, &c->d_omega_bar, 1))) return s;
    if ((s = dalloc(c, &c->d_partial, 1024))) return s;
    const size_t ne = (size_t)d.nc + 2 * GH;
    if ((s = dalloc(c, &c->d_extb, (size_t)12 * d.chunk * ne * ne * ne))) return s;
    if ((s = dalloc(c, &c->d.ftr_b, (size_t)d.fd_cap * 6 * 12 * d.np1 * d.np1))) return s;
    const size_t fch = (size_t)(d.chunk < FDV_CHUNK ? d.chunk : FDV_CHUNK);
    if ((s = dalloc(c, &c->d_gbuf, (size_t)3 * 12 * fch * (d.nc + 1) * d.nc * d.nc * 6))) return s;
    c->adj_ready = true;
    return FFE_OK;
}

// out = filter (or its transpose) of in on DG elements; FD blocks are copied
static ffe_status filter_or_copy(ffe_ctx* c, Field in, Field out, int transpose) {
    const Dev& d = c->d;
    if (d.filter_on) {
        launch_filter(d, in, out, NV, transpose, c->st);
        if (c->adj_fd)
            CK(cudaMemcpyAsync(out.fd(0), in.fd(0), (size_t)NV * d.nfd * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    } else {
        CK(cudaMemcpyAsync(out.p, in.p, (size_t)NV * (d.ndg + (c->adj_fd ? d.nfd : 0)) * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->st));
    }
    return FFE_OK;
}

// right-hand side of the hybrid operator at U (fixed mask)
static void rhs_at(ffe_ctx* c, Field U, Field out) {
    const Dev& d = c->d;
    if (c->adj_fd) launch_current(d, U, c->J, nullptr, 0, c->st);
    launch_dg_substep_curved(d, SUB_RHS, U, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, out, out, c->G1,
                             c->st);
    if (c->adj_fd)
        launch_fd_substep(d, SUB_RHS, d.fd_list, 1, U, c->J, c->un, c->F2, c->F3, c->G1, c->G2, c->G3, c->G4, out, out,
                          c->G1, c->st);
}

// out = (d RHS/dU)^T L at U for the hybrid operator (fixed mask)
static void rhs_vjp_at(ffe_ctx* c, Field U, Field L, Field out) {
    const Dev& d = c->d;
    cudaMemsetAsync(out.fd(0), 0, (size_t)NV * d.nfd * sizeof(double), c->st);
    launch_rhs_vjp(d, U, L, out, c->d_omega_bar, c->st);
    if (c->adj_fd) {
        launch_fd_traces_vjp(d, U, out, c->st);
        launch_current(d, U, c->J, nullptr, 0, c->st);
        launch_fd_rhs_vjp(d, U, c->J, L, out, c->d_extb, c->d_gbuf, c->d_omega_bar, c->st);
    }
}

ffe_status ffe_rhs_vjp(ffe_ctx* c, const double* U_dev, const double* lam_dev, double* out_dev, double* omega_bar) try {
    g_err.clear();
    if (!c || !U_dev || !lam_dev || !out_dev) return fail(FFE_EINVAL, "null argument");
    ffe_status s;
    if ((s = adjoint_ready(c))) return s;
    const Dev& d = c->d;
    Field U{(double*)U_dev, NV, d.ndg, d.nfd}, L{(double*)lam_dev, NV, d.ndg, d.nfd}, O{out_dev, NV, d.ndg, d.nfd};
    CK(cudaMemsetAsync(c->d_omega_bar, 0, sizeof(double), c->st));
    launch_build_lists(d, c->st);
    rhs_vjp_at(c, U, L, O);
    prof_collect(c->st);
    if (omega_bar) {
        double ob = 0.0;
        CK(cudaMemcpyAsync(&ob, c->d_omega_bar, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        *omega_bar += ob;
    }
    CK(cudaGetLastError());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

// Forward recomputation of a step's stages from U_n (a.un): stage s = 3, 4 is
// R_s (explicit part) -> T_s = filter(R_s) -> U_s = S(T_s), G_s = G(U_s).  With
// next, also u_{n+1} = filter(W), W the explicit part of the last substep.
static ffe_status adj_forward(ffe_ctx* c, AdjArgs& a, const Field* next) {
    const Dev& d = c->d;
    cudaStream_t st = c->st;
    ffe_status s;
    launch_adj(d, 0, a, 0, st);
    rhs_at(c, a.U2, a.F2);
    launch_adj(d, 1, a, SUB_A, st);
    if ((s = filter_or_copy(c, a.R3, a.T3, 0))) return s;
    launch_adj(d, 6, a, SUB_A, st);
    rhs_at(c, a.U3, a.F3);
    launch_adj(d, 1, a, SUB_B, st);
    if ((s = filter_or_copy(c, a.R4, a.T4, 0))) return s;
    launch_adj(d, 6, a, SUB_B, st);
    rhs_at(c, a.U4, a.F4);
    if (next) {
        launch_adj(d, 1, a, SUB_C, st);
        if ((s = filter_or_copy(c, a.W, *next, 0))) return s;
        if (d.mode != FFE_RELAX) launch_adj_clamp(d, *next, st);
    }
    return FFE_OK;
}

// Reverse sweep of one step given its stages (a.un, a.U2, a.T3, a.U3, a.T4, a.U4).
static ffe_status adj_reverse(ffe_ctx* c, AdjArgs& a, Field lin, double* omega_bar) {
    const Dev& d = c->d;
    cudaStream_t st = c->st;
    ffe_status s;
    CK(cudaMemsetAsync(c->d_omega_bar, 0, sizeof(double), st));
    if (d.mode != FFE_RELAX) {
        // u_{n+1} = clamp(X), X = filter(W): back through the clamp at X
        launch_adj(d, 1, a, SUB_C, st);                                 // W
        if ((s = filter_or_copy(c, a.W, a.tmp2, 0))) return s;          // X
        launch_adj_clamp_back(d, a.tmp2, lin, a.ubar, st);              // X-bar (ubar is free until the seeds)
        if ((s = filter_or_copy(c, a.ubar, a.tmp, 1))) return s;        // W-bar
    } else if ((s = filter_or_copy(c, lin, a.tmp, 1))) {                // W-bar (u_{n+1} = filter(W))
        return s;
    }
    launch_adj(d, 2, a, 0, st);                                         // seeds
    rhs_vjp_at(c, a.U4, a.F4b, a.tmp);                                  // U4-bar from F4
    launch_adj_addG(d, a.U4, a.G4b, a.tmp, st);                         // + G4 = G(U4)
    launch_adj(d, 5, a, SUB_B, st);                                     // T4-bar (tmp2)
    if ((s = filter_or_copy(c, a.tmp2, a.tmp, 1))) return s;            // R4-bar (tmp)
    launch_adj(d, 3, a, SUB_B, st);
    rhs_vjp_at(c, a.U3, a.F3b, a.tmp);
    launch_adj_addG(d, a.U3, a.G3b, a.tmp, st);
    launch_adj(d, 5, a, SUB_A, st);                                     // T3-bar
    if ((s = filter_or_copy(c, a.tmp2, a.tmp, 1))) return s;            // R3-bar
    launch_adj(d, 3, a, SUB_A, st);
    rhs_vjp_at(c, a.U2, a.F2b, a.tmp);
    launch_adj_addG(d, a.U2, a.G2b, a.tmp, st);                         // U2-bar
    launch_adj(d, 4, a, 0, st);                                         // stages 2, 1 -> lambda_n
    prof_collect(st);
    if (omega_bar) {
        double ob = 0.0;
        CK(cudaMemcpyAsync(&ob, c->d_omega_bar, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *omega_bar += ob;
    }
    CK(cudaGetLastError());
    return FFE_OK;
}

// the five stored stages of a step: [U2][T3][U3][T4][U4], state vectors
static void point_stages(const Dev& d, AdjArgs& a, double* stages) {
    const int64_t n = (int64_t)NV * (d.ndg + d.nfd);
    Field* f[5] = {&a.U2, &a.T3, &a.U3, &a.T4, &a.U4};
    for (int i = 0; i < 5; ++i) *f[i] = Field{stages + i * n, NV, d.ndg, d.nfd};
}

ffe_status ffe_adjoint_step(ffe_ctx* c, const double* U_dev, const double* lam_in_dev, double* lam_out_dev,
                            double* omega_bar) try {
    g_err.clear();
    if (!c || !U_dev || !lam_in_dev || !lam_out_dev) return fail(FFE_EINVAL, "null argument");
    ffe_status s;
    if ((s = adjoint_ready(c))) return s;
    const Dev& d = c->d;
    AdjArgs a = c->adj;
    a.un = Field{(double*)U_dev, NV, d.ndg, d.nfd};
    a.lam = Field{lam_out_dev, NV, d.ndg, d.nfd};
    launch_build_lists(d, c->st);
    if ((s = adj_forward(c, a, nullptr))) return s;
    return adj_reverse(c, a, Field{(double*)lam_in_dev, NV, d.ndg, d.nfd}, omega_bar);
} catch (...) {
    return host_failure();
}

ffe_status ffe_adjoint_forward(ffe_ctx* c, const double* U_dev, double* stages_dev, double* U_next_dev) try {
    g_err.clear();
    if (!c || !U_dev) return fail(FFE_EINVAL, "null argument");
    if (U_next_dev == U_dev) return fail(FFE_EINVAL, "U_next must not alias U");
    ffe_status s;
    if ((s = adjoint_ready(c))) return s;
    const Dev& d = c->d;
    AdjArgs a = c->adj;
    a.un = Field{(double*)U_dev, NV, d.ndg, d.nfd};
    if (stages_dev) point_stages(d, a, stages_dev);
    launch_build_lists(d, c->st);
    Field next{U_next_dev, NV, d.ndg, d.nfd};
    if ((s = adj_forward(c, a, U_next_dev ? &next : nullptr))) return s;
    CK(cudaGetLastError());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_adjoint_reverse(ffe_ctx* c, const double* U_dev, const double* stages_dev, const double* lam_in_dev,
                               double* lam_out_dev, double* omega_bar) try {
    g_err.clear();
    if (!c || !U_dev || !stages_dev || !lam_in_dev || !lam_out_dev) return fail(FFE_EINVAL, "null argument");
    ffe_status s;
    if ((s = adjoint_ready(c))) return s;
    const Dev& d = c->d;
    AdjArgs a = c->adj;
    a.un = Field{(double*)U_dev, NV, d.ndg, d.nfd};
    a.lam = Field{lam_out_dev, NV, d.ndg, d.nfd};
    launch_build_lists(d, c->st);
    if (d.mode != FFE_RELAX) {
        // the clamp at the step's end needs the pre-clamp state, built from the
        // step's right-hand sides, which the stored stages do not hold: recompute
        // the step in the context's own stage fields (the stored ones stay untouched)
        if ((s = adj_forward(c, a, nullptr))) return s;
    } else {
        point_stages(d, a, (double*)stages_dev);
    }
    return adj_reverse(c, a, Field{(double*)lam_in_dev, NV, d.ndg, d.nfd}, omega_bar);
} catch (...) {
    return host_failure();
}

ffe_status ffe_luminosity(ffe_ctx* c, const double* U_dev, double r_L, double* L_host, double* grad_dev,
                          double scale) try {
    g_err.clear();
    if (!c || !U_dev) return fail(FFE_EINVAL, "null argument");
    if (c->batch) return fail(FFE_ENOTIMPL, "ffe_luminosity takes single contexts (batches: ffe_diagnostic)");
    int inst, na;
    ffe_status s;
    if ((s = surface_target(c, nullptr, r_L, &inst, &na))) return s;
    const ffe_ctx::Surf* sf;
    if ((s = surface_get(c, r_L, false, -1, &sf))) return s;
    return surface_sum(c, *sf, U_dev, 0, grad_dev, scale, L_host);
} catch (...) {
    return host_failure();
}

ffe_status ffe_initial_tangent(ffe_ctx* c, int which, double* dU_dev) try {
    g_err.clear();
    if (!c || !dU_dev) return fail(FFE_EINVAL, "null argument");
    if (c->id_kind != FFE_ID_DIPOLE || c->batch) return fail(FFE_ENOTIMPL, "tangents are built for the dipole data");
    if (which != 0 && which != 2) return fail(FFE_EINVAL, "dipole parameter %d has no tangent (0 = mu, 2 = chi)", which);
    const Dev& d = c->d;
    const double mu = c->id_prm.size() > 0 ? c->id_prm[0] : 1.0;
    const double dl = c->id_prm.size() > 1 ? c->id_prm[1] : 0.1;
    const double chi = c->id_prm.size() > 2 ? c->id_prm[2] : 0.0;
    std::vector<double> xdg(3 * (size_t)d.ndg), T(NV * (size_t)(d.ndg + d.nfd), 0.0);
    std::vector<unsigned char> mask(d.E);
    CK(cudaMemcpy(xdg.data(), d.xyz_dg, xdg.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(mask.data(), d.mask, d.E, cudaMemcpyDeviceToHost));
    // B = mu [3 x (m.x) - m (r^2 - 2 delta^2)] / (r^2 + delta^2)^(5/2), m = (sin chi, 0, cos chi)
    const double m[3] = {std::sin(chi), 0.0, std::cos(chi)}, dm[3] = {std::cos(chi), 0.0, -std::sin(chi)};
    auto tangent_B = [&](const double* x, double* tb) {
        const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        const double f = 1.0 / std::pow(r2 + dl * dl, 2.5);
        const double* mm = which == 0 ? m : dm;
        const double scale = which == 0 ? 1.0 : mu;
        const double mx = mm[0] * x[0] + mm[1] * x[1] + mm[2] * x[2];
        for (int i = 0; i < 3; ++i) tb[i] = scale * f * (3.0 * x[i] * mx - mm[i] * (r2 - 2.0 * dl * dl));
    };
    // DG nodes of DG elements
    parallel_for(d.ndg, [&](int64_t p) {
        if (mask[p / d.nn]) return;
        const double x[3] = {xdg[p], xdg[d.ndg + p], xdg[2 * d.ndg + p]};
        double tb[3];
        tangent_B(x, tb);
        for (int i = 0; i < 3; ++i) T[(3 + i) * d.ndg + p] = tb[i];
    });
    // cells of FD elements (their data is the initial data at the cell centres)
    MapFn map = ctx_map(c);
    parallel_for(d.E, [&](int64_t e) {
        if (!mask[e]) return;
        const int nc = d.nc;
        const int64_t base = (int64_t)(d.fd_slot ? c->h_fd_slot[e] : e) * d.ncell;
        for (int q = 0; q < nc * nc * nc; ++q) {
            const int cc[3] = {q % nc, (q / nc) % nc, q / (nc * nc)};
            double xi[3], X[3], ij[3][3], tb[3];
            for (int a = 0; a < 3; ++a) xi[a] = -1.0 + (cc[a] + 0.5) * 2.0 / nc;
            map((int)e, xi, X, ij);
            tangent_B(X, tb);
            for (int i = 0; i < 3; ++i) T[NV * d.ndg + (3 + i) * d.nfd + base + q] = tb[i];
        }
    });
    CK(cudaMemcpy(dU_dev, T.data(), T.size() * 8, cudaMemcpyHostToDevice));
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_set_profiling(ffe_ctx* c, int on) try {
    if (!c) return fail(FFE_EINVAL, "null context");
    CK(cudaStreamSynchronize(c->st));
    g_prof.on = on != 0;
    g_prof.pending.clear();
    g_prof.used = 0;
    return FFE_OK;
} catch (...) {
    return host_failure();
}

ffe_status ffe_profile_read(ffe_ctx* c, char* buf, size_t cap) try {
    if (!c || !buf || cap == 0) return fail(FFE_EINVAL, "bad argument");
    std::string js = "{";
    for (size_t i = 0; i < g_prof.totals.size(); ++i) {
        char tmp[160];
        snprintf(tmp, sizeof tmp, "%s\"%s\": [%ld, %.6f, %.6f]", i ? ", " : "", g_prof.totals[i].first.c_str(),
                 g_prof.totals[i].second.n, g_prof.totals[i].second.ms, g_prof.totals[i].second.max_ms);
        js += tmp;
    }
    js += "}";
    g_prof.totals.clear();
    snprintf(buf, cap, "%s", js.c_str());
    return FFE_OK;
} catch (...) {
    return host_failure();
}

void ffe_destroy(ffe_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

}  // extern "C"
