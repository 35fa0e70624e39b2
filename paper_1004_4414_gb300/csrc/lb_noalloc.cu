// lb_noalloc.cu -- lb_field_moments: field sums of a population array that
// the caller already holds on the device, computed without allocating.
//
// Some callers cannot allocate device memory at the point where they want
// these sums: a monitor that runs between the steps of a long job must not
// call cudaMalloc or cudaFree, because those can synchronise the whole
// device (stalling the job's other streams) and can fail outright once the
// job has committed nearly all of the device memory to its boxes.  So this
// entry point takes its scratch from a fixed array that is part of the
// loaded library (a file-scope __device__ array, present on every device
// that loads the library until the process exits) and asks the caller only
// for the input fields and an output buffer.
//
// The sums are the same ones lb_observables forms from a handle's state
// (k_obs_partial / k_obs_final): per-component mass, total fluid momentum,
// the largest fluid speed |j|/rho and the fluid and solid node counts.

#include <mutex>

#include "lbpart.h"
#include "lb_common.cuh"

namespace lbp {
namespace {

constexpr int FM_W = 8;          // values per partial, in the output order
constexpr int FM_THREADS = 256;  // threads per block; the scratch holds one partial per block

// Scratch: one partial of FM_W doubles per block (256 KB in all).  Every
// call writes the partials of the blocks it launches before its final pass
// reads them, so nothing here has to start at zero; the contents left by
// one call are simply overwritten by the next.
__device__ __align__(256) double g_fm_scratch[LB_FIELD_MOMENTS_MAX_BLOCKS * FM_W];

// The blocks sum the nodes of f[2][19][N] grid-stride (block b takes nodes
// b * FM_THREADS + t + k * gridDim.x * FM_THREADS), so a small field still
// spreads over many blocks; owner[n] != -1 marks a solid node, whose
// populations are ignored.
__global__ void __launch_bounds__(FM_THREADS) k_fm_partial(const double* __restrict__ f,
                                                           const int32_t* __restrict__ owner, int64_t N,
                                                           double* __restrict__ partials) {
    double v[FM_W] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t step = (int64_t)gridDim.x * FM_THREADS;
    for (int64_t n = (int64_t)blockIdx.x * FM_THREADS + threadIdx.x; n < N; n += step) {
        if (owner[n] != -1) {
            v[7] += 1.0;
            continue;
        }
        double rt = 0, jt[3] = {0, 0, 0};
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < 19; i++) {
                const double x = f[((int64_t)c * 19 + i) * N + n];
                v[c] += x;
                rt += x;
                jt[0] += x * cx(i);
                jt[1] += x * cy(i);
                jt[2] += x * cz(i);
            }
        v[2] += jt[0];
        v[3] += jt[1];
        v[4] += jt[2];
        v[5] = fmax(v[5], sqrt(jt[0] * jt[0] + jt[1] * jt[1] + jt[2] * jt[2]) / rt);
        v[6] += 1.0;
    }
    __shared__ double s[FM_THREADS / 32][FM_W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < FM_W; k++) {
        double x = v[k];
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_xor_sync(0xffffffffu, x, off);
            x = (k == 5) ? fmax(x, o) : x + o;
        }
        if (lane == 0) s[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < FM_W) {
        const int k = threadIdx.x;
        double x = s[0][k];
        for (int w = 1; w < FM_THREADS / 32; w++) x = (k == 5) ? fmax(x, s[w][k]) : x + s[w][k];
        partials[(int64_t)blockIdx.x * FM_W + k] = x;
    }
}

// One warp: out[k] = combination over the nblocks partials (max for k = 5).
__global__ void k_fm_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= FM_W) return;
    double x = 0.0;
    for (int b = 0; b < nblocks; b++) {
        const double y = partials[b * FM_W + k];
        x = (k == 5) ? fmax(x, y) : x + y;
    }
    out[k] = x;
}

// Device address of the scratch array, looked up once per device.
constexpr int FM_MAX_DEVICES = 64;
std::mutex g_fm_mutex;
double* g_fm_ptr[FM_MAX_DEVICES] = {};

int scratch_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LB_ECUDA;
    if (dev < 0 || dev >= FM_MAX_DEVICES) return LB_EINVAL;
    std::lock_guard<std::mutex> lock(g_fm_mutex);
    if (!g_fm_ptr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_fm_scratch) != cudaSuccess || !p) return LB_ECUDA;
        g_fm_ptr[dev] = p;
    }
    *out = g_fm_ptr[dev];
    return LB_OK;
}

// A pointer the kernels may dereference on the current device: device or
// managed memory, suitably aligned.
bool device_pointer_ok(const void* p, size_t align) {
    if (!p || ((uintptr_t)p % align) != 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess && a.device == dev;
}

}  // namespace
}  // namespace lbp

extern "C" int lb_field_moments(const double* d_f, const int32_t* d_owner, int64_t n_nodes, void* stream,
                                double* d_out) {
    using namespace lbp;
    if (n_nodes < 0 || n_nodes > (int64_t)LB_FIELD_MOMENTS_MAX_NODES) return LB_EINVAL;
    if (!device_pointer_ok(d_out, sizeof(double))) return LB_EINVAL;
    if (n_nodes > 0 && (!device_pointer_ok(d_f, sizeof(double)) || !device_pointer_ok(d_owner, sizeof(int32_t))))
        return LB_EINVAL;
    double* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != LB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // one block per FM_THREADS nodes, at most the scratch's partials
    const int64_t want = (n_nodes + FM_THREADS - 1) / FM_THREADS;
    const int nblocks = (int)(want < LB_FIELD_MOMENTS_MAX_BLOCKS ? want : LB_FIELD_MOMENTS_MAX_BLOCKS);
    if (nblocks > 0) k_fm_partial<<<nblocks, FM_THREADS, 0, st>>>(d_f, d_owner, n_nodes, scratch);
    k_fm_final<<<1, 32, 0, st>>>(scratch, nblocks, d_out);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}
