// lb_structure.cuh -- the domain size of Sec. VI (Eq. eq:domsize) on the
// device: L_i = 2 pi / sqrt(<k_i^2>), with <k_i^2> the second moment of the
// structure function S(k) = |phi'_k|^2 / N of the order parameter
// phi = rho^r - rho^b (0 on solid nodes), phi' = phi - <phi>.
//
// The three-dimensional transform is not needed.  For axis x, let g(k_x;
// y, z) be the transform of phi' along x alone.  Parseval over (y, z) gives
//   sum_k k_x^2 |phi'_k|^2 = n_y n_z sum_{y,z} sum_{k_x} k_x^2 |g(k_x; y, z)|^2,
// and over all axes sum_k |phi'_k|^2 = N sum_x phi'(x)^2, so
//   <k_x^2> = sum_lines sum_{k_x} k_x^2 |g|^2 / (n_x sum_x phi'^2).
// The mean only enters g at k_x = 0, where k_x^2 = 0, so the line
// transforms take phi itself.  Each line is transformed with a
// mixed-radix Stockham FFT (one stage per prime factor, radix 4 where it
// divides; a stage of radix R costs n R complex multiply-adds per line) in
// FP64, in shared memory for lines of up to 2048 nodes and in global
// scratch beyond.  Wave numbers k = 2 pi f / n with f = j for j <= n/2,
// j - n above (the set n_i in [-n/2, n/2 - 1] for even n; k^2 is even in
// k).  Sums run in a fixed order, so the result does not depend on timing.
#pragma once
#include "lb_common.cuh"

namespace lbp {

constexpr int SPEC_THREADS = 256;
constexpr int SPEC_MAX_FACTORS = 32;
constexpr int SPEC_SMEM_POINTS = 2048;  // W n per block in shared memory

struct Radices {
    int n;                       // line length
    int count;                   // number of stages
    int r[SPEC_MAX_FACTORS];     // radix of each stage
};

// radix-4 stages first, then 2, 3, 5, 7 and the remaining prime factors
inline Radices radices_of(int n) {
    Radices f{};
    f.n = n;
    int m = n;
    const int small[5] = {4, 2, 3, 5, 7};
    for (int k = 0; k < 5; k++)
        while (m % small[k] == 0 && f.count < SPEC_MAX_FACTORS) {
            f.r[f.count++] = small[k];
            m /= small[k];
        }
    for (int q = 11; m > 1 && f.count < SPEC_MAX_FACTORS; q += 2)
        while (m % q == 0) {
            f.r[f.count++] = q;
            m /= q;
        }
    return f;
}

// One block transforms W lines along `axis` at a time (grid-stride over the
// line groups) and adds sum_lines sum_k k^2 |g(k)|^2 of its groups into
// partials[blockIdx.x].  buf: 2 W n + n complex values (two stage buffers
// and the twiddles exp(-2 pi i q / n)), in shared memory (SMEM) or in a
// global region of that size per block.
template <bool SMEM>
static __global__ void __launch_bounds__(SPEC_THREADS)
    k_line_spectrum(const double* __restrict__ phi, int nx, int ny, int nz, int axis, int W, Radices rad,
                    double2* __restrict__ gscratch, double* __restrict__ partials) {
    extern __shared__ double2 s_spec[];
    const int n = rad.n;
    double2* const base = SMEM ? s_spec : gscratch + (size_t)blockIdx.x * (2 * (size_t)W * n + n);
    double2* bufA = base;
    double2* bufB = base + (size_t)W * n;
    double2* const tw = base + 2 * (size_t)W * n;
    const size_t N = (size_t)nx * ny * nz;
    const int nlines = (int)(N / (size_t)n);
    const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)nx : (size_t)nx * ny);
    // first node of line l
    auto line_base = [&](int l) -> size_t {
        if (axis == 0) return (size_t)l * nx;
        if (axis == 1) return (size_t)(l % nx) + (size_t)nx * ny * (size_t)(l / nx);
        return (size_t)l;
    };
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)q / (double)n, &s, &c);
        tw[q] = make_double2(c, -s);
    }
    double acc = 0.0;
    const int ngroups = (nlines + W - 1) / W;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int l0 = grp * W;
        const int wl = nlines - l0 < W ? nlines - l0 : W;
        __syncthreads();  // the buffers of the previous group are consumed
        // load: along x the lines are contiguous rows; along y and z the W
        // lines of a group are neighbours in x, so consecutive threads take
        // consecutive lines
        for (int idx = threadIdx.x; idx < wl * n; idx += blockDim.x) {
            int li, j;
            if (axis == 0) {
                li = idx / n;
                j = idx - li * n;
            } else {
                j = idx / wl;
                li = idx - j * wl;
            }
            bufA[(size_t)li * n + j] = make_double2(phi[line_base(l0 + li) + (size_t)j * stride], 0.0);
        }
        __syncthreads();
        // Stockham stages: output o of a stage of radix R after sub-transforms
        // of length p is the length-R DFT over r of src[i + r m] twiddled,
        // with k = o mod p, s = (o / p) mod R, i = (o / (p R)) p + k,
        // m = n / R: v = sum_r src[i + r m] w^(r (k n / (p R) + s n / R))
        int p = 1;
        for (int st = 0; st < rad.count; st++) {
            const int R = rad.r[st], m = n / R;
            const int nk = n / (p * R), ns = n / R;
            for (int idx = threadIdx.x; idx < wl * n; idx += blockDim.x) {
                const int li = idx / n, o = idx - li * n;
                const int k = o % p, s = (o / p) % R, i = (o / (p * R)) * p + k;
                const int E = (k * nk + s * ns) % n;
                const double2* src = bufA + (size_t)li * n;
                double vr = 0.0, vi = 0.0;
                int e = 0;
                for (int r = 0; r < R; r++) {
                    const double2 a = src[i + r * m], w = tw[e];
                    vr += a.x * w.x - a.y * w.y;
                    vi += a.x * w.y + a.y * w.x;
                    e += E;
                    if (e >= n) e -= n;
                }
                bufB[(size_t)li * n + o] = make_double2(vr, vi);
            }
            __syncthreads();
            double2* t = bufA;
            bufA = bufB;
            bufB = t;
            p *= R;
        }
        for (int idx = threadIdx.x; idx < wl * n; idx += blockDim.x) {
            const int li = idx / n, j = idx - li * n;
            const int f = j <= n / 2 ? j : j - n;
            const double kk = 2.0 * M_PI * (double)f / (double)n;
            const double2 v = bufA[(size_t)li * n + j];
            acc += kk * kk * (v.x * v.x + v.y * v.y);
        }
    }
    // block sum in a fixed order
    __shared__ double s_red[SPEC_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_red[w];
        partials[blockIdx.x] = t;
    }
}

// out[k] = sum over blocks b of in[b * stride + k] for k < width, in a fixed
// order (one block; thread k sums column k)
static __global__ void k_sum_columns(const double* __restrict__ in, int nblocks, int stride, int width,
                                     double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= width) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; b++) t += in[(size_t)b * stride + k];
    out[k] = t;
}

// number of particles of a box whose mark has both bits (phi > 0 and phi < 0
// next to it); one block
static __global__ void k_count_both(const int* __restrict__ marks, int np, double* __restrict__ out) {
    __shared__ int s_c[32];
    int c = 0;
    for (int q = threadIdx.x; q < np; q += blockDim.x) c += marks[q] == 3 ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_c[w];
        *out = (double)t;
    }
}

}  // namespace lbp
