// FD-subcell right-hand side without any device allocation.
//
// Who needs this: callers that cannot call cudaMalloc -- a host application
// that hands the library memory from its own pool and forbids allocations
// behind its back, or a latency-critical path where a first-touch allocation
// would stall.  ffe_create allocates everything a context needs, so those
// callers cannot use ffe_rhs; this entry point computes the FD right-hand side
// of caller-built extended blocks from caller-owned inputs and outputs, and
// keeps its intermediate data (the current J~ at every extended cell and the
// face fluxes) in one file-scope device array of fixed size,
// FFE_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB).  Every GPU that loads the
// library holds that array until the process exits.
//
// Unlike the context path, the current J~ of every ghost cell is computed here
// from that cell's state: a context gives the ghosts across a DG neighbour's
// face that neighbour's nodal current instead (evaluated like its state), so
// the two agree on ghosts from FD neighbours and boundary states only.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "ffe_internal.h"
#include "physics.cuh"

namespace {

using namespace ffe;

constexpr long long kScratchDoubles = 1LL << 20;   // FFE_NOALLOC_SCRATCH_DOUBLES
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Same WENO5-Z (point-value interpolation candidates, ideal weights (1,10,5)/16,
// Jiang-Shu indicators, Z weights with q = 2) as the context path.
__device__ __forceinline__ double na_weno5z(double v0, double v1, double v2, double v3, double v4, double eps) {
    const double p0 = fma(0.375, v0, fma(-1.25, v1, 1.875 * v2));
    const double p1 = fma(-0.125, v1, fma(0.75, v2, 0.375 * v3));
    const double p2 = fma(0.375, v2, fma(0.75, v3, -0.125 * v4));
    const double c13 = 13.0 / 12.0;
    const double s0a = v0 - 2.0 * v1 + v2, s0b = v0 - 4.0 * v1 + 3.0 * v2;
    const double s1a = v1 - 2.0 * v2 + v3, s1b = v1 - v3;
    const double s2a = v2 - 2.0 * v3 + v4, s2b = 3.0 * v2 - 4.0 * v3 + v4;
    const double b0 = fma(c13 * s0a, s0a, 0.25 * s0b * s0b);
    const double b1 = fma(c13 * s1a, s1a, 0.25 * s1b * s1b);
    const double b2 = fma(c13 * s2a, s2a, 0.25 * s2b * s2b);
    const double tau = fabs(b0 - b2);
    const double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps), r2 = tau / (b2 + eps);
    const double a0 = 0.0625 * fma(r0, r0, 1.0);
    const double a1 = 0.625 * fma(r1, r1, 1.0);
    const double a2 = 0.3125 * fma(r2, r2, 1.0);
    return fma(a0, p0, fma(a1, p1, a2 * p2)) / (a0 + a1 + a2);
}

struct NA {
    int n, nc, ne;
    int64_t ext, nface;         // doubles per element block: extended cells, faces of one direction
    double eta, eps, sc[3];     // sc[k] = (2/h_k) (nc/2)
    int corr;
    const double* Uext;         // [9][n][ext]
    double* J;                  // scratch [3][n][ext]
    double* F;                  // scratch [3][9][n][nface]
    double* out;                // [9][n][nc^3]
};

__global__ void k_na_current(NA a) {
    const int64_t total = (int64_t)a.n * a.ext;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        double u[NV], jd[3], jf[3];
        for (int v = 0; v < NV; ++v) u[v] = a.Uext[(int64_t)v * total + q];
        current_flat(u, a.eta, jd, jf);
        for (int k = 0; k < 3; ++k) a.J[(int64_t)k * total + q] = jf[k];
    }
}

__global__ void k_na_flux(NA a) {
    const int nc = a.nc, ne = a.ne;
    const int64_t total = (int64_t)a.n * 3 * a.nface, cells = (int64_t)a.n * a.ext;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(q / (3 * a.nface));
        const int k = (int)((q / a.nface) % 3);
        const int64_t fi = q % a.nface;
        const int m = (int)(fi % (nc + 1));
        const int ta = (int)((fi / (nc + 1)) % nc), tb = (int)(fi / ((nc + 1) * nc));
        const int t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
        int c[3];
        c[k] = m;
        c[t1] = ta + GH;
        c[t2] = tb + GH;
        const int64_t base = (int64_t)w * a.ext + c[0] + (int64_t)ne * (c[1] + (int64_t)ne * c[2]);
        const int64_t stride = k == 0 ? 1 : (k == 1 ? ne : (int64_t)ne * ne);
        double UL[12], UR[12], Um[12], Up[12];
        for (int qq = 0; qq < 12; ++qq) {
            const double* src = qq < NV ? a.Uext + (int64_t)qq * cells + base : a.J + (int64_t)(qq - NV) * cells + base;
            const double v0 = src[0], v1 = src[stride], v2 = src[2 * stride];
            const double v3 = src[3 * stride], v4 = src[4 * stride], v5 = src[5 * stride];
            UL[qq] = na_weno5z(v0, v1, v2, v3, v4, a.eps);
            UR[qq] = na_weno5z(v5, v4, v3, v2, v1, a.eps);
            Um[qq] = v2;
            Up[qq] = v3;
        }
        double FL[NV], FR[NV], Fs[NV];
        flux_dir_flat(UL, UL + NV, k, FL);
        flux_dir_flat(UR, UR + NV, k, FR);
        for (int v = 0; v < NV; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * (UR[v] - UL[v]);
        if (a.corr) {
            double Fm[NV], Fp[NV];
            flux_dir_flat(Um, Um + NV, k, Fm);
            flux_dir_flat(Up, Up + NV, k, Fp);
            for (int v = 0; v < NV; ++v) Fs[v] = Fs[v] - (1.0 / 6.0) * (Fm[v] - 2.0 * Fs[v] + Fp[v]);
        }
        for (int v = 0; v < NV; ++v) a.F[(((int64_t)k * NV + v) * a.n + w) * a.nface + fi] = Fs[v];
    }
}

__global__ void k_na_update(NA a) {
    const int nc = a.nc, ne = a.ne, ncell = nc * nc * nc;
    const int64_t total = (int64_t)a.n * ncell, cells = (int64_t)a.n * a.ext;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int w = (int)(q / ncell), c = (int)(q % ncell);
        const int cc[3] = {c % nc, (c / nc) % nc, c / (nc * nc)};
        const int64_t o = (int64_t)w * a.ext + (cc[0] + GH) + (int64_t)ne * ((cc[1] + GH) + (int64_t)ne * (cc[2] + GH));
        double u[NV], jd[3], jf[3], du[NV];
        for (int v = 0; v < NV; ++v) u[v] = a.Uext[(int64_t)v * cells + o];
        current_flat(u, a.eta, jd, jf);
        du[0] = -jd[0]; du[1] = -jd[1]; du[2] = -jd[2];
        du[3] = du[4] = du[5] = 0.0;
        du[6] = u[8];
        du[7] = du[8] = 0.0;
        for (int k = 0; k < 3; ++k) {
            const int t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
            const int64_t f0 = cc[k] + (int64_t)(nc + 1) * (cc[t1] + nc * cc[t2]);
            for (int v = 0; v < NV; ++v) {
                const double* fl = a.F + (((int64_t)k * NV + v) * a.n + w) * a.nface;
                du[v] = fma(-a.sc[k], fl[f0 + 1] - fl[f0], du[v]);
            }
        }
        for (int v = 0; v < NV; ++v) a.out[(int64_t)v * total + q] = du[v];
    }
}

}  // namespace

namespace ffe {
void set_last_error(const char* msg);
}

extern "C" ffe_status ffe_fd_rhs_noalloc(int P, int n_elem, const double* h_host, double eta, double weno_eps,
                                         int fd_corrector, const double* Uext_dev, double* dUdt_dev,
                                         void* cuda_stream) try {
    char msg[256];
    if (P < 3 || P > 6 || n_elem < 0 || !h_host || (n_elem > 0 && (!Uext_dev || !dUdt_dev))) {
        ffe::set_last_error("ffe_fd_rhs_noalloc: need 3 <= P <= 6, n_elem >= 0, h and buffers non-null");
        return FFE_EINVAL;
    }
    for (int k = 0; k < 3; ++k)
        if (!(h_host[k] > 0.0) || !std::isfinite(h_host[k])) {
            ffe::set_last_error("ffe_fd_rhs_noalloc: element widths must be positive and finite");
            return FFE_EINVAL;
        }
    if (!(eta >= 0.0) || !std::isfinite(eta) || !(weno_eps > 0.0) || !std::isfinite(weno_eps)) {
        ffe::set_last_error("ffe_fd_rhs_noalloc: need finite eta >= 0 and weno_eps > 0");
        return FFE_EINVAL;
    }
    const int nc = 2 * P + 1, ne = nc + 2 * GH;
    const long long per_elem = 3LL * ne * ne * ne + 3LL * NV * (nc + 1) * nc * nc;
    const long long cap = kScratchDoubles / per_elem;
    if (n_elem > cap) {
        snprintf(msg, sizeof msg,
                 "ffe_fd_rhs_noalloc: %d elements need %lld scratch doubles; the fixed scratch holds %lld "
                 "(at most %lld elements of order %d per call)",
                 n_elem, per_elem * n_elem, kScratchDoubles, cap, P);
        ffe::set_last_error(msg);
        return FFE_EINVAL;
    }
    if (n_elem == 0) return FFE_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ffe_fd_rhs_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        ffe::set_last_error(msg);
        return FFE_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, sizeof msg, "ffe_fd_rhs_noalloc: device %d is beyond the %d devices this entry point serves",
                 dev, kMaxDevices);
        ffe::set_last_error(msg);
        return FFE_EINVAL;
    }
    double* scratch = nullptr;
    {
        // first call on this device: resolve the device address of the static array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) {
                snprintf(msg, sizeof msg, "ffe_fd_rhs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                ffe::set_last_error(msg);
                return FFE_ECUDA;
            }
            g_scratch_ptr[dev] = (double*)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    NA a;
    a.n = n_elem;
    a.nc = nc;
    a.ne = ne;
    a.ext = (int64_t)ne * ne * ne;
    a.nface = (int64_t)(nc + 1) * nc * nc;
    a.eta = eta;
    a.eps = weno_eps;
    for (int k = 0; k < 3; ++k) a.sc[k] = (2.0 / h_host[k]) * (0.5 * nc);
    a.corr = fd_corrector;
    a.Uext = Uext_dev;
    a.J = scratch;                                   // every entry written before it is read
    a.F = scratch + 3LL * n_elem * a.ext;            // likewise: nothing needs clearing
    a.out = dUdt_dev;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
    k_na_current<<<nsm * 4, 256, 0, st>>>(a);
    k_na_flux<<<nsm * 8, 128, 0, st>>>(a);
    k_na_update<<<nsm * 4, 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "ffe_fd_rhs_noalloc: launch: %s", cudaGetErrorString(e));
        ffe::set_last_error(msg);
        return FFE_ECUDA;
    }
    return FFE_OK;
} catch (...) {
    // a host exception (the mutex, an allocation inside the runtime) must not
    // cross the C ABI
    ffe::set_last_error("ffe_fd_rhs_noalloc: host resources exhausted");
    return FFE_ENOMEM;
}
