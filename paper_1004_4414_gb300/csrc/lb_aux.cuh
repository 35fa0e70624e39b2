// lb_aux.cuh -- kernels outside the time step: node status from particle
// positions, initial populations, canonical export / import of the state,
// densities, and the observables reduction.
#pragma once
#include "lb_common.cuh"
#include "lb_particles.cuh"

namespace lbp {

template <class T>
static __global__ void k_fill(T* __restrict__ p, T v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// Claim of the nodes inside each particle (sphere or spheroid, inside_shape)
// for a state with no previous status: pass 1 keeps the smallest squared
// centre distance per node (FP64 bits, which order like the values for
// non-negative numbers), pass 2 the lowest particle index among the
// particles at that distance.
template <int PASS>
static __global__ void k_claim(const BoxDev* __restrict__ boxes, Shared sh, int b, unsigned long long* __restrict__ key,
                        int* __restrict__ idbuf) {
    const BoxDev& B = boxes[b];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lp = blockIdx.x * (blockDim.x >> 5) + wib;
    if (lp >= B.np) return;
    const int p = B.pstart + lp;
    const PartState ps = sh.part[p];
    const double R = B.rb;
    const int dims[3] = {B.nx, B.ny, B.nz};
    int lo[3], span[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = (int)floor(ps.X[a] - R);
        span[a] = (int)floor(ps.X[a] + R) - lo[a] + 1;
        if (span[a] > dims[a]) span[a] = dims[a];
    }
    const int total = span[0] * span[1] * span[2];
    for (int idx = lane; idx < total; idx += 32) {
        const int kx = idx % span[0], ky = (idx / span[0]) % span[1], kz = idx / (span[0] * span[1]);
        const int gx = wrapi(lo[0] + kx, B.nx), gy = wrapi(lo[1] + ky, B.ny), gz = wrapi(lo[2] + kz, B.nz);
        const double dx = mimg((double)gx - ps.X[0], B.nx), dy = mimg((double)gy - ps.X[1], B.ny),
                     dz = mimg((double)gz - ps.X[2], B.nz);
        if (!inside_shape(B, dx, dy, dz, ps.E)) continue;
        const double d2 = dist2_nc(dx, dy, dz);
        const int n = gx + B.nx * (gy + B.ny * gz);
        if (B.owner[n] == OWN_WALL) continue;
        const unsigned long long k = (unsigned long long)__double_as_longlong(d2);
        if (PASS == 1) atomicMin(&key[n], k);
        else if (key[n] == k) atomicMin(&idbuf[n], p);
    }
}

static __global__ void k_owner_from_claims(const BoxDev* __restrict__ boxes, int b, const int* __restrict__ idbuf) {
    const BoxDev& B = boxes[b];
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        if (B.owner[n] == OWN_WALL) {
            B.flags[n] = FL_SOLID;
            continue;
        }
        const int id = idbuf[n];
        B.owner[n] = id == 0x7fffffff ? OWN_FLUID : id;
        B.flags[n] = id == 0x7fffffff ? 0 : FL_SOLID;
    }
}

static __global__ void k_shell_all(const BoxDev* __restrict__ boxes, int b) {
    const BoxDev& B = boxes[b];
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) shell_update(B, n);
}

// Owner map of one box from the caller (box-local particle indices) into
// global indices in out; bit 1 of *flags: an entry outside [-2, np), bit 2:
// a static wall node.
static __global__ void k_owner_import(const int32_t* __restrict__ in, int32_t* __restrict__ out, int N, int np,
                                      int pstart, int* flags) {
    int bad = 0, wall = 0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int o = in[n];
        if (o >= np || o < -2) bad = 1;
        if (o == OWN_WALL) wall = 1;
        out[n] = o >= 0 ? o + pstart : o;
    }
    bad = __any_sync(0xffffffffu, bad);
    wall = __any_sync(0xffffffffu, wall);
    if ((threadIdx.x & 31) == 0 && (bad | wall)) atomicOr(flags, bad | (wall << 1));
}

// box-local owner map for export: particle indices minus the box's first
static __global__ void k_owner_export(const int32_t* __restrict__ in, int32_t* __restrict__ out, int N, int pstart) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int o = in[n];
        out[n] = o >= 0 ? o - pstart : o;
    }
}

// owner map given by the caller (global particle indices already applied)
static __global__ void k_flags_from_owner(const BoxDev* __restrict__ boxes, int b) {
    const BoxDev& B = boxes[b];
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x)
        B.flags[n] = B.owner[n] == OWN_FLUID ? 0 : FL_SOLID;
}

// f = f^eq(rho, u) on fluid nodes in the even-step layout (own slots);
// rho from a field [2][N] (canonical order) or from SplitMix64 noise; u
// from a field [3][N] or zero.  The density ring slot rc ([N][2] pairs)
// gets rho on fluid nodes, 0 elsewhere.
template <class P>
static __global__ void k_init_pop(const BoxDev* __restrict__ boxes, int b, const double* __restrict__ rho_field,
                           const double* __restrict__ u_field, uint64_t s_red, uint64_t s_blue, double noise,
                           int rc, double* __restrict__ mass_out) {
    using R = typename P::real;
    const BoxDev& B = boxes[b];
    const Pop<P> pop(B);
    R* rcur = reinterpret_cast<R*>(B.rho[rc]);
    double m0 = 0.0, m1 = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        if (B.flags[n] & FL_SOLID) {
            rcur[2 * (size_t)n] = R(0);
            rcur[2 * (size_t)n + 1] = R(0);
            continue;
        }
        double rho[2];
        if (rho_field) {
            rho[0] = rho_field[n];
            rho[1] = rho_field[(size_t)B.N + n];
        } else {
            // noise U(-a, a): output n of the red / blue noise streams
            rho[0] = B.rho_init[0] + noise * (2.0 * sm64_unit(s_red, (uint64_t)n) - 1.0);
            rho[1] = B.rho_init[1] + noise * (2.0 * sm64_unit(s_blue, (uint64_t)n) - 1.0);
        }
        const R ux = u_field ? (R)u_field[n] : R(0);
        const R uy = u_field ? (R)u_field[(size_t)B.N + n] : R(0);
        const R uz = u_field ? (R)u_field[(size_t)2 * B.N + n] : R(0);
        for (int c = 0; c < 2; c++) {
            const R r = (R)rho[c];
            R resid = R(0), sent = R(0);
            for (int i = 1; i < 19; i++) {
                const R fe = feq_rt<R>(i, r, ux, uy, uz);
                const R q = pop.store(c, i, n, fe);
                resid += fe - q;
                sent += q;
            }
            // the rest population: rho minus the 18 stored values, kept only
            // as part of the density
            sent += feq_rest<R>(r, ux, uy, uz) + resid;
            rcur[2 * (size_t)n + c] = sent;
            if (c == 0) m0 += (double)sent;
            else m1 += (double)sent;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        m0 += __shfl_xor_sync(0xffffffffu, m0, off);
        m1 += __shfl_xor_sync(0xffffffffu, m1, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&mass_out[0], m0);
        atomicAdd(&mass_out[1], m1);
    }
}

// populations of node n at the coming step of parity par: before an even
// step f_i sits in slot i of n, before an odd step in slot opp(i) of n - c_i
// (whatever the status of n - c_i)
template <class P>
__device__ __forceinline__ typename P::real load_node_pop(const BoxDev& B, const Pop<P>& pop, int par, int c, int i,
                                                          int n) {
    if (par == 0 || i == 0) return pop.load(c, i, n);
    return pop.load(c, opp(i), nbr_index(B, n, -cx(i), -cy(i), -cz(i)));
}

// f_0 of a fluid node: its density (ring slot rc) minus the 18 moving
// populations, in double
template <class P>
__device__ __forceinline__ double rest_of(const BoxDev& B, const Pop<P>& pop, int par, int rc, int c, int n) {
    using R = typename P::real;
    double s = 0.0;
#pragma unroll
    for (int i = 1; i < 19; i++) s += (double)load_node_pop<P>(B, pop, par, c, i, n);
    return (double)reinterpret_cast<const R*>(B.rho[rc])[2 * (size_t)n + c] - s;
}

// direction i of both components of box b in canonical order: out[c * N + n]
// (0 on solid nodes; for i = 0 the rest population rho^c - sum_{i>0} f_i)
template <class P>
static __global__ void k_export_dir(const BoxDev* __restrict__ boxes, int b, int i, int par, int rc,
                                    double* __restrict__ out) {
    using R = typename P::real;
    const BoxDev& B = boxes[b];
    const Pop<P> pop(B);
    const size_t N = (size_t)B.N;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        double v0 = 0.0, v1 = 0.0;
        if (!(B.flags[n] & FL_SOLID)) {
            if (i == 0) {
                v0 = rest_of<P>(B, pop, par, rc, 0, n);
                v1 = rest_of<P>(B, pop, par, rc, 1, n);
            } else {
                // before an even step f_i sits in slot i of n, before an odd
                // step in slot opp(i) of n - c_i
                const int slot = par == 0 ? i : opp(i);
                const int m = par == 0 ? n : nbr_index(B, n, -cx(i), -cy(i), -cz(i));
                R a, c;
                pop.ld2(pop.pair(slot, m), i, a, c);
                v0 = (double)a;
                v1 = (double)c;
            }
        }
        out[n] = v0;
        out[N + n] = v1;
    }
}

// direction i of both components from canonical order in[c * N + n]
template <class P>
static __global__ void k_import_dir(const BoxDev* __restrict__ boxes, int b, int i, int par,
                                    const double* __restrict__ in) {
    using R = typename P::real;
    const BoxDev& B = boxes[b];
    const Pop<P> pop(B);
    const size_t N = (size_t)B.N;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        if (B.flags[n] & FL_SOLID) continue;
        const R v0 = (R)in[n], v1 = (R)in[N + n];
        if (i == 0) {
            pop.store(0, 0, n, v0);
            pop.store(1, 0, n, v1);
        } else {
            const int slot = par == 0 ? i : opp(i);
            const int m = par == 0 ? n : nbr_index(B, n, -cx(i), -cy(i), -cz(i));
            R q0, q1;
            pop.st2(pop.pair(slot, m), i, v0, v1, q0, q1);
        }
    }
}

// rho^c on fluid nodes (0 on solid) into ring slot rc and/or a double
// array; fluid mass into mass_out.  With src < 0 rho^c = sum_i f_i of
// freshly imported populations (rest slot included), else the density
// field of ring slot src.
template <class P>
static __global__ void k_rho_from_pop(const BoxDev* __restrict__ boxes, int b, int par, int src, int rc,
                                      double* __restrict__ out, double* __restrict__ mass_out) {
    using R = typename P::real;
    const BoxDev& B = boxes[b];
    const Pop<P> pop(B);
    R* rcur = rc >= 0 ? reinterpret_cast<R*>(B.rho[rc]) : nullptr;
    const R* rsrc = src >= 0 ? reinterpret_cast<const R*>(B.rho[src]) : nullptr;
    double m0 = 0.0, m1 = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        R r[2] = {R(0), R(0)};
        if (!(B.flags[n] & FL_SOLID))
            for (int c = 0; c < 2; c++) {
                if (rsrc) r[c] = rsrc[2 * (size_t)n + c];
                else
                    for (int i = 0; i < 19; i++) r[c] += load_node_pop<P>(B, pop, par, c, i, n);
            }
        if (rcur) {
            rcur[2 * (size_t)n] = r[0];
            rcur[2 * (size_t)n + 1] = r[1];
        }
        if (out) {
            out[n] = (double)r[0];
            out[(size_t)B.N + n] = (double)r[1];
        }
        m0 += (double)r[0];
        m1 += (double)r[1];
    }
    if (mass_out) {
        for (int off = 16; off > 0; off >>= 1) {
            m0 += __shfl_xor_sync(0xffffffffu, m0, off);
            m1 += __shfl_xor_sync(0xffffffffu, m1, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&mass_out[0], m0);
            atomicAdd(&mass_out[1], m1);
        }
    }
}

// ------------------------------------------------------------ observables
// Per block: mass[2], fluid momentum[3], max |u|, fluid and solid node
// counts -> partials[block][8]; a second single-block pass reduces them.
constexpr int OBS_W = 8;
constexpr int OBS_BLOCKS = 304;
// The mass of a fluid node is its density (ring slot rc); the momentum
// comes from the 18 moving populations.
template <class P>
static __global__ void __launch_bounds__(256) k_obs_partial(const BoxDev* __restrict__ boxes, int b, int par, int rc,
                                                            double* __restrict__ partials) {
    using R = typename P::real;
    const BoxDev& B = boxes[b];
    const Pop<P> pop(B);
    const R* __restrict__ rho = reinterpret_cast<const R*>(B.rho[rc]);
    double v[OBS_W] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        if (B.flags[n] & FL_SOLID) {
            v[7] += 1.0;
            continue;
        }
        double rt = 0, jt[3] = {0, 0, 0};
        for (int c = 0; c < 2; c++) {
            const double r = (double)rho[2 * (size_t)n + c];
            v[c] += r;
            rt += r;
            for (int i = 1; i < 19; i++) {
                const double f = (double)load_node_pop<P>(B, pop, par, c, i, n);
                jt[0] += f * cx(i);
                jt[1] += f * cy(i);
                jt[2] += f * cz(i);
            }
        }
        v[2] += jt[0];
        v[3] += jt[1];
        v[4] += jt[2];
        const double um = sqrt(jt[0] * jt[0] + jt[1] * jt[1] + jt[2] * jt[2]) / rt;
        v[5] = fmax(v[5], um);
        v[6] += 1.0;
    }
    __shared__ double s[8][OBS_W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < OBS_W; k++) {
        double x = v[k];
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_xor_sync(0xffffffffu, x, off);
            x = (k == 5) ? fmax(x, o) : x + o;
        }
        if (lane == 0) s[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < OBS_W) {
        const int k = threadIdx.x;
        double x = s[0][k];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) x = (k == 5) ? fmax(x, s[w][k]) : x + s[w][k];
        partials[blockIdx.x * OBS_W + k] = x;
    }
}

// Order parameter phi = rho^r - rho^b on fluid nodes, 0 on solid nodes
// (Sec. VI), into phi[N] (canonical order, may be NULL), and per-block sums
// of phi and phi^2 into partials[block][2] (fixed order within the block).
template <class P>
static __global__ void __launch_bounds__(256) k_phi(const BoxDev* __restrict__ boxes, int b, int rc,
                                                    double* __restrict__ phi, double* __restrict__ partials) {
    using R = typename P::real;
    using R2 = typename Real2<R>::type;
    const BoxDev& B = boxes[b];
    const R2* __restrict__ r2 = rpair<R>(B.rho[rc]);
    double s0 = 0.0, s1 = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (!(B.flags[n] & FL_SOLID)) {
            const R2 r = r2[n];
            v = (double)r.x - (double)r.y;
        }
        if (phi) phi[n] = v;
        s0 += v;
        s1 += v * v;
    }
    __shared__ double s_r[8][2];
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_r[threadIdx.x >> 5][0] = s0;
        s_r[threadIdx.x >> 5][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_r[w][threadIdx.x];
        partials[blockIdx.x * 2 + threadIdx.x] = t;
    }
}

// Interface coverage marks (the paper names the covered interface but
// does not define it; the reading here): for every solid node of a particle
// q of box b, the fluid D3Q19 neighbours with phi > 0 set bit 1 and those
// with phi < 0 bit 2 of marks[q - pstart].  A particle covers the interface
// when both bits are set.
template <class P>
static __global__ void k_coverage_marks(const BoxDev* __restrict__ boxes, int b, int rc, int* __restrict__ marks) {
    using R = typename P::real;
    using R2 = typename Real2<R>::type;
    const BoxDev& B = boxes[b];
    const R2* __restrict__ r2 = rpair<R>(B.rho[rc]);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        const int o = B.owner[n];
        if (o < B.pstart || o >= B.pstart + B.np) continue;
        int bits = 0, x, y, z;
        node_xyz(B, n, x, y, z);
#pragma unroll
        for (int i = 1; i < 19; i++) {
            const int m = node_off(B, x, y, z, cx(i), cy(i), cz(i));
            if (B.flags[m] & FL_SOLID) continue;
            const R2 r = r2[m];
            const double v = (double)r.x - (double)r.y;
            if (v > 0.0) bits |= 1;
            else if (v < 0.0) bits |= 2;
        }
        if (bits) atomicOr(&marks[o - B.pstart], bits);
    }
}

static __global__ void k_obs_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= OBS_W) return;
    double x = 0.0;
    for (int i = 0; i < nblocks; i++) x = (k == 5) ? fmax(x, partials[i * OBS_W + k]) : x + partials[i * OBS_W + k];
    out[k] = x;
}

}  // namespace lbp
