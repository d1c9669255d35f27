// Quasi-random loading of an ellipsoid bunch (manual Sec. "Electron Bunch Generation": Halton
// numbers, Eqs. uniform1D, gaussian1D, gaussian2D; the Gaussian edges that keep a uniform current
// profile from radiating coherently at its ends; the bunching factor, Eq. bunchingFactor, and the
// shot noise, Eq. negativeExponential, applied to the lab positions).  One thread per particle:
// every particle's Halton numbers follow from its index alone.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "../../include/mithra.h"
#include "common.cuh"
#include "kernels.h"
#include "run.h"

namespace mithra {
namespace {

__constant__ unsigned kPrimes[20] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71};

// One minus the radical inverse of j in base kPrimes[i] (the digits of j mirrored about the
// radix point), with every operation rounded separately so that the value is the same
// correctly rounded sequence of operations on any IEEE machine.
__device__ __forceinline__ double halton(int i, unsigned j)
{
    const unsigned p = kPrimes[i];
    const double dp = (double)p;
    double x = 0.0, scale = __ddiv_rn(1.0, dp);
    while (j > 0) {
        x = __dadd_rn(x, __dmul_rn((double)(j % p), scale));
        j /= p;
        scale = __ddiv_rn(scale, dp);
    }
    return __dsub_rn(1.0, x);
}

struct EllArgs {
    mithra_ellipsoid e;
    int64_t n, nu;     // particles, of which nu fill the flat part of a uniform profile
    double uz0;        // sqrt(gamma^2 - 1)
    unsigned j0;       // Halton index offset
};

// Bases (the manual leaves the assignment open): 2,3 transverse positions (Eq. gaussian2D), 5,7
// transverse momenta, 11 (13) the longitudinal position (Eq. uniform1D / gaussian1D), 17,19 the
// longitudinal momentum spread; particle p at index p + 1 + j0.
__global__ void k_ellipsoid(EllArgs a, double* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    const mithra_ellipsoid& e = a.e;
    const unsigned j = (unsigned)(p + 1) + a.j0;
    double* q = out + 6 * p;
    const double r1 = sqrt(-2.0 * log(halton(0, j))), a1 = 2.0 * kPi * halton(1, j);
    q[0] = e.sig[0] * r1 * cos(a1);
    q[1] = e.sig[1] * r1 * sin(a1);
    const double r2 = sqrt(-2.0 * log(halton(2, j))), a2 = 2.0 * kPi * halton(3, j);
    q[3] = e.sig_u[0] * r2 * cos(a2);
    q[4] = e.sig_u[1] * r2 * sin(a2);
    double z;
    if (!e.uniform) {
        z = e.sig[2] * sqrt(-2.0 * log(halton(4, j))) * cos(2.0 * kPi * halton(5, j));
    } else if (p < a.nu) {
        z = 2.0 * e.sig[2] * (halton(4, j) - 0.5);
    } else {
        // Gaussian edges of the same peak line density: lower half to the tail, upper half to
        // the head of the flat part
        const unsigned je = (unsigned)(p - a.nu + 1) + a.j0;
        const double ze = e.cse_sigma * sqrt(-2.0 * log(halton(4, je))) * cos(2.0 * kPi * halton(5, je));
        z = ze < 0.0 ? -e.sig[2] + ze : e.sig[2] + ze;
    }
    if (e.lambda_r > 0.0 && e.bunching > 0.0) {
        const double k = 2.0 * kPi / e.lambda_r;
        z -= (2.0 * e.bunching / k) * sin(k * z + e.bunching_phase);
    }
    q[2] = z;
    q[5] = a.uz0 + e.sig_u[2] * sqrt(-2.0 * log(halton(6, j))) * cos(2.0 * kPi * halton(7, j));
}

// Shot noise: slice s = floor(z / lambda_r) - s0 of every particle, its count, then the
// modulation with amplitude sqrt(-2 ln x_s) / sqrt(N_e,s) and phase 2 pi y_s (bases 23, 29 at
// index s + 1), N_e,s = charge_e n_s / n.
__global__ void k_slice_range(const double* __restrict__ out, int64_t n, double lam, long long* __restrict__ mm)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const long long s = (long long)floor(out[6 * p + 2] / lam);
    atomicMin(mm, s);
    atomicMax(mm + 1, s);
}

__global__ void k_slice_count(const double* __restrict__ out, int64_t n, double lam, long long s0,
                              unsigned* __restrict__ cnt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    atomicAdd(cnt + ((long long)floor(out[6 * p + 2] / lam) - s0), 1u);
}

__global__ void k_shot_noise(double* __restrict__ out, int64_t n, double lam, long long s0, double charge_e,
                             const unsigned* __restrict__ cnt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double* z = out + 6 * p + 2;
    const long long s = (long long)floor(*z / lam) - s0;
    const double ne = charge_e * (double)cnt[s] / (double)n;
    const double b = sqrt(-2.0 * log(halton(8, (unsigned)(s + 1)))) / sqrt(ne);
    const double ph = 2.0 * kPi * halton(9, (unsigned)(s + 1));
    const double k = 2.0 * kPi / lam;
    *z -= (2.0 * b / k) * sin(k * *z + ph);
}

}  // namespace
}  // namespace mithra

using mithra::set_last_error;

int mithra::ellipsoid_device(const mithra_ellipsoid& ell, int64_t n, uint64_t j0, double* d, void* (*alloc)(void*, size_t),
                             void (*free_fn)(void*, void*), void* ctx, cudaStream_t st)
{
    using namespace mithra;
    const mithra_ellipsoid* e = &ell;
    for (double v : {e->gamma, e->sig[0], e->sig[1], e->sig[2], e->sig_u[0], e->sig_u[1], e->sig_u[2], e->cse_sigma,
                     e->lambda_r, e->bunching, e->bunching_phase, e->charge_e})
        if (!std::isfinite(v)) return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: non-finite value");
    if (!(e->gamma >= 1.0)) return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: gamma must be >= 1");
    if (e->shot_noise && !(e->lambda_r > 0.0 && e->charge_e > 0.0))
        return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: shot noise needs lambda_r > 0 and charge_e > 0");
    if (n < 0 || (uint64_t)n + j0 >= ((uint64_t)1 << 32) - 1)
        return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: n + seed out of range");
    if (n == 0) return MITHRA_OK;
    EllArgs a;
    a.e = *e;
    a.n = n;
    a.nu = n;
    a.j0 = (unsigned)j0;
    const double L = 2.0 * e->sig[2];
    if (e->uniform && e->cse_sigma > 0.0) a.nu = (int64_t)std::llround((double)n * L / (L + std::sqrt(2.0 * kPi) * e->cse_sigma));
    a.uz0 = std::sqrt(e->gamma * e->gamma - 1.0);
    int rc = MITHRA_OK;
    long long* mm = nullptr;
    unsigned* cnt = nullptr;
    const unsigned nb = (unsigned)((n + 255) / 256);
    do {
        k_ellipsoid<<<nb, 256, 0, st>>>(a, d);
        count_launches(1);
        if (e->shot_noise) {
            if (!(mm = (long long*)alloc(ctx, 2 * sizeof(long long)))) {
                rc = set_last_error(MITHRA_ENOMEM, "ellipsoid_bunch: device allocation failed");
                break;
            }
            const long long init[2] = {LLONG_MAX, LLONG_MIN};
            if (cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, st) != cudaSuccess) break;
            k_slice_range<<<nb, 256, 0, st>>>(d, n, e->lambda_r, mm);
            long long h[2];
            if (cudaMemcpyAsync(h, mm, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                break;
            const long long ns = h[1] - h[0] + 1;
            if (ns < 1 || ns > ((long long)1 << 31)) {
                rc = set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: too many shot-noise slices");
                break;
            }
            if (!(cnt = (unsigned*)alloc(ctx, (size_t)ns * sizeof(unsigned)))) {
                rc = set_last_error(MITHRA_ENOMEM, "ellipsoid_bunch: device allocation failed");
                break;
            }
            if (cudaMemsetAsync(cnt, 0, (size_t)ns * sizeof(unsigned), st) != cudaSuccess) break;
            k_slice_count<<<nb, 256, 0, st>>>(d, n, e->lambda_r, h[0], cnt);
            k_shot_noise<<<nb, 256, 0, st>>>(d, n, e->lambda_r, h[0], e->charge_e, cnt);
            count_launches(3);
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) break;
    } while (false);
    const cudaError_t err = cudaGetLastError();
    if (rc == MITHRA_OK && err != cudaSuccess) rc = set_last_error(MITHRA_ECUDA, cudaGetErrorString(err));
    if (cudaStreamSynchronize(st) != cudaSuccess) cudaGetLastError();
    if (cnt) free_fn(ctx, cnt);
    if (mm) free_fn(ctx, mm);
    return rc;
}

namespace {
struct HostAlloc {
    mithra_alloc_fn af;
    mithra_free_fn ff;
    void* ctx;
};
void* host_alloc(void* c, size_t b)
{
    auto* h = (HostAlloc*)c;
    if (h->af) return h->af(h->ctx, b);
    void* p = nullptr;
    if (cudaMalloc(&p, b) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void host_free(void* c, void* p)
{
    auto* h = (HostAlloc*)c;
    if (!p) return;
    if (h->ff) h->ff(h->ctx, p);
    else cudaFree(p);
}
}  // namespace

extern "C" int mithra_ellipsoid_bunch(const mithra_ellipsoid* e, int64_t n, double* out6, void* stream)
{
    using namespace mithra;
    if (!e || (n > 0 && !out6)) return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: null argument");
    if (n < 0 || n >= ((int64_t)1 << 32) - 1) return set_last_error(MITHRA_EINVAL, "ellipsoid_bunch: n out of range");
    if (n == 0) return ellipsoid_device(*e, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    HostAlloc ha;
    get_allocator(&ha.af, &ha.ff, &ha.ctx);
    double* d = (double*)host_alloc(&ha, (size_t)n * 6 * sizeof(double));
    if (!d) return set_last_error(MITHRA_ENOMEM, "ellipsoid_bunch: device allocation failed");
    int rc = ellipsoid_device(*e, n, 0, d, host_alloc, host_free, &ha, st);
    if (rc == MITHRA_OK) {
        if (cudaMemcpyAsync(out6, d, (size_t)n * 6 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            const cudaError_t err = cudaGetLastError();
            rc = set_last_error(MITHRA_ECUDA, cudaGetErrorString(err));
        }
    }
    host_free(&ha, d);
    return rc;
}
