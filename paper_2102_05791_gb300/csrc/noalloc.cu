// sim_energy_noalloc: the energy E(x, a) of a mesh held entirely in
// caller-owned device arrays, evaluated without allocating any device
// memory.
//
// Some callers cannot call cudaMalloc when they need an energy value: a
// process whose GPU memory has been claimed up front by another framework's
// pool allocator, or code that must not allocate once its setup is done.
// This entry point needs no handle (building a handle allocates) and keeps
// its only scratch -- one FP64 partial sum per block, the block counter of
// the final reduction and a count of invalid rest elements -- in a fixed-size
// array that lives in the library
// image.  Every GPU that loads the library holds that array (about 33 KB)
// until the process exits.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before capturing a stream.  All calls share the array and it
// keeps the last call's contents, so calls that overlap on the GPU (on
// different streams, or from different host threads) race; serialise them.
// A rest element with non-positive area or volume makes the mesh invalid:
// the call then waits for its stream, finds the element count the kernel
// recorded, and returns SIM_EINVERTED (E_out holds NaN).
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "reduce.cuh"
#include "softsim.h"

namespace {

constexpr int kNoAllocBlocks = 4096;     // maximum grid of the energy kernel
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPerBlock = 1024;   // elements (and vertices) per block
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    double partial[kNoAllocBlocks];
    unsigned int ticket;      // blocks done (last-block reduction)
    unsigned int n_inverted;  // rest elements with non-positive measure
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local std::string g_noalloc_error;
thread_local unsigned int g_inverted_host;  // read-back target of the inverted-element count

struct NoAllocMaterial {
    double mu, lam, k, rho, grav, kc;
    int cpow, log_mode, muscle;
};

// Energy of element e from rest and current positions: W (Psi + psi_m), with
// psi_m = k/2 a |F f|^2 (contractile) or k/2 (|F f|/a - 1)^2 (active spring),
// plus the element's share of the gravity potential, rho W g / (dim+1) * sum y.
template <int D>
__device__ double element_energy(int64_t e, const double *X, const int32_t *T, const double *x, const double *a,
                                 const double *fiber, const NoAllocMaterial &m, unsigned int *n_inverted)
{
    const int32_t *t = T + e * (D + 1);
    double Dm[D][D], Ds[D][D];
    for (int k = 0; k < D; ++k)
        for (int i = 0; i < D; ++i) {
            Dm[i][k] = X[(int64_t)t[k + 1] * D + i] - X[(int64_t)t[0] * D + i];
            Ds[i][k] = x[(int64_t)t[k + 1] * D + i] - x[(int64_t)t[0] * D + i];
        }
    double Bi[D][D], det;
    if constexpr (D == 2) {
        det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
        Bi[0][0] = Dm[1][1] / det;
        Bi[0][1] = -Dm[0][1] / det;
        Bi[1][0] = -Dm[1][0] / det;
        Bi[1][1] = Dm[0][0] / det;
    } else {
        double C[3][3];
        for (int j = 0; j < 3; ++j) {
            const int p = (j + 1) % 3, q = (j + 2) % 3;
            C[0][j] = Dm[1][p] * Dm[2][q] - Dm[2][p] * Dm[1][q];
            C[1][j] = Dm[2][p] * Dm[0][q] - Dm[0][p] * Dm[2][q];
            C[2][j] = Dm[0][p] * Dm[1][q] - Dm[1][p] * Dm[0][q];
        }
        det = Dm[0][0] * C[0][0] + Dm[1][0] * C[1][0] + Dm[2][0] * C[2][0];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Bi[i][j] = C[j][i] / det;
    }
    if (!(det > 0.0)) {  // inverted rest element: the mesh is invalid
        atomicAdd(n_inverted, 1u);
        return NAN;
    }
    const double W = det / (D == 2 ? 2.0 : 6.0);
    double F[D][D];
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += Ds[i][k] * Bi[k][j];
            F[i][j] = s;
        }
    double J;
    if constexpr (D == 2)
        J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    else
        J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
            F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    double I1 = 0.0, Ff2 = 0.0;
    for (int i = 0; i < D; ++i) {
        double ff = 0.0;
        for (int j = 0; j < D; ++j) {
            I1 += F[i][j] * F[i][j];
            ff += F[i][j] * fiber[e * D + j];
        }
        Ff2 += ff * ff;
    }
    double l;
    if (m.log_mode == SIM_LOG_EXACT) {
        if (J <= 0.0) return INFINITY;  // a NaN J (non-finite input) stays NaN
        l = log(J);
    } else {
        l = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
    }
    double ysum = 0.0;
    for (int k = 0; k <= D; ++k) ysum += x[(int64_t)t[k] * D + 1];
    double psim = 0.5 * m.k * a[e] * Ff2;
    if (m.muscle) {
        const double r = sqrt(Ff2) / a[e] - 1.0;
        psim = 0.5 * m.k * r * r;
    }
    return W * (0.5 * m.mu * (I1 - D) - m.mu * l + 0.5 * m.lam * l * l + psim) +
           m.rho * W * m.grav / (D + 1) * ysum;
}

template <int D>
__global__ void __launch_bounds__(kNoAllocThreads)
    k_energy_noalloc(int64_t nv, int64_t ne, const double *__restrict__ X, const int32_t *__restrict__ T,
                     const double *__restrict__ x, const double *__restrict__ a, const double *__restrict__ fiber,
                     NoAllocMaterial m, NoAllocScratch *__restrict__ scratch, double *__restrict__ E_out)
{
    double s = 0.0;
    const int64_t b0 = (int64_t)blockIdx.x * kNoAllocPerBlock;
    for (int64_t e = b0 + threadIdx.x; e < ne && e < b0 + kNoAllocPerBlock; e += blockDim.x)
        s += element_energy<D>(e, X, T, x, a, fiber, m, &scratch->n_inverted);
    for (int64_t i = b0 + threadIdx.x; i < nv && i < b0 + kNoAllocPerBlock; i += blockDim.x) {
        const double y = x[i * D + 1];
        const double pen = y < 0.0 ? -y : 0.0;
        s += m.kc * (m.cpow == 2 ? pen * pen : pen * pen * pen);
    }
    const double bs = softsim::block_sum(s);
    if (threadIdx.x == 0) scratch->partial[blockIdx.x] = bs;
    if (softsim::last_block(&scratch->ticket, gridDim.x)) {
        const double tot = softsim::sum_partials(scratch->partial, gridDim.x);
        if (threadIdx.x == 0) *E_out = tot;
    }
}

int noalloc_fail(int code, const std::string &msg)
{
    g_noalloc_error = msg;
    return code;
}

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(NoAllocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(SIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SIM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(SIM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_ptr[dev];
    return SIM_OK;
}

}  // namespace

extern "C" const char *sim_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" int sim_energy_noalloc(int dim, int64_t n_vert, int64_t n_elem, const double *rest_pos,
                                  const int32_t *elems, const double *x, const double *a, const double *fiber,
                                  const sim_material *mat, double *E_out, void *stream)
{
    if (dim != 2 && dim != 3) return noalloc_fail(SIM_EINVAL, "dim must be 2 or 3");
    if (n_vert <= 0 || n_elem <= 0 || !rest_pos || !elems || !x || !a || !fiber || !mat || !E_out)
        return noalloc_fail(SIM_EINVAL, "null or empty argument");
    const int64_t cap = (int64_t)kNoAllocBlocks * kNoAllocPerBlock;
    if (n_elem > cap || n_vert > cap)
        return noalloc_fail(SIM_EINVAL, "mesh too large for sim_energy_noalloc: at most " + std::to_string(cap) +
                                            " elements and vertices");
    if (mat->contact_power != 2 && mat->contact_power != 3)
        return noalloc_fail(SIM_EINVAL, "contact_power must be 2 or 3");
    if (mat->log_mode != SIM_LOG_EXACT && mat->log_mode != SIM_LOG_QUAD)
        return noalloc_fail(SIM_EINVAL, "log_mode must be SIM_LOG_EXACT or SIM_LOG_QUAD");
    if (mat->muscle_model != SIM_MUSCLE_CONTRACTILE && mat->muscle_model != SIM_MUSCLE_SPRING)
        return noalloc_fail(SIM_EINVAL, "muscle_model must be SIM_MUSCLE_CONTRACTILE or SIM_MUSCLE_SPRING");
    NoAllocScratch *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != SIM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the block counter and the inverted-element count must start at zero;
    // the partial sums are all overwritten
    cudaError_t e = cudaMemsetAsync(&scratch->ticket, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return noalloc_fail(SIM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const NoAllocMaterial m{mat->mu, mat->lambda, mat->k_muscle, mat->density, mat->gravity, mat->k_contact,
                            mat->contact_power, mat->log_mode, mat->muscle_model};
    const int64_t nmax = n_elem > n_vert ? n_elem : n_vert;
    const int grid = (int)((nmax + kNoAllocPerBlock - 1) / kNoAllocPerBlock);
    if (dim == 2)
        k_energy_noalloc<2><<<grid, kNoAllocThreads, 0, s>>>(n_vert, n_elem, rest_pos, elems, x, a, fiber, m, scratch,
                                                             E_out);
    else
        k_energy_noalloc<3><<<grid, kNoAllocThreads, 0, s>>>(n_vert, n_elem, rest_pos, elems, x, a, fiber, m, scratch,
                                                             E_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(SIM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    // the status depends on the rest mesh: read the kernel's count (pageable
    // host target, no allocation) and wait for the stream
    e = cudaMemcpyAsync(&g_inverted_host, &scratch->n_inverted, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(SIM_ECUDA, std::string("read-back: ") + cudaGetErrorString(e));
    if (g_inverted_host != 0)
        return noalloc_fail(SIM_EINVERTED, std::to_string(g_inverted_host) +
                                               " rest element(s) with non-positive area or volume; E is NaN");
    return SIM_OK;
}
