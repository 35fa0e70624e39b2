// lb_particles.cuh -- particle-side kernels of one time step: cell list and
// neighbour list, remap of the spheres onto the lattice (cover / uncover,
// Sec. III and Sec. IV), the virtual fluid of the shell with particle colour
// (Sec. IV), and the MD update with Hertz contact and lubrication (Sec. III).
//
// All kernels work on the particles of every box at once (one launch per
// phase for the whole batch); a particle knows its box through pbox[].
#pragma once
#include "lb_common.cuh"
#include "lb_step_kernel.cuh"

namespace lbp {

// ------------------------------------------------------------ cell list
__device__ __forceinline__ int cell_of(const BoxDev& B, const double X[3]) {
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int v = (int)(X[a] / B.cell_len[a]);
        c[a] = v < 0 ? 0 : (v >= B.nc[a] ? B.nc[a] - 1 : v);
    }
    return B.cell_off + c[0] + B.nc[0] * (c[1] + B.nc[1] * c[2]);
}

static __global__ void k_step_begin(const BoxDev* __restrict__ boxes, int nb, Shared sh, int total_cells, int mslot_next) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = tid; i < total_cells; i += gridDim.x * blockDim.x) sh.cell_count[i] = 0;
    if (tid == 0) *sh.ev_count = 0;
    if (tid < nb) {
        boxes[tid].mass_acc[mslot_next * 2 + 0] = 0.0;
        boxes[tid].mass_acc[mslot_next * 2 + 1] = 0.0;
    }
}

static __global__ void k_cell_count(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    atomicAdd(&sh.cell_count[cell_of(B, sh.part[p].X)], 1);
}

// one block per box: exclusive scan of the cell counts (offset by the box's
// first particle), cursors = starts
static __global__ void k_cell_scan(const BoxDev* __restrict__ boxes, Shared sh) {
    const BoxDev& B = boxes[blockIdx.x];
    const int ncell = B.nc[0] * B.nc[1] * B.nc[2];
    __shared__ int s_tmp[1024];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = B.pstart;
    __syncthreads();
    for (int base = 0; base < ncell; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < ncell ? sh.cell_count[B.cell_off + i] : 0;
        s_tmp[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < blockDim.x; off <<= 1) {
            int t = threadIdx.x >= off ? s_tmp[threadIdx.x - off] : 0;
            __syncthreads();
            s_tmp[threadIdx.x] += t;
            __syncthreads();
        }
        const int incl = s_tmp[threadIdx.x];
        if (i < ncell) {
            const int st = s_carry + incl - v;
            sh.cell_start[B.cell_off + i] = st;
            sh.cell_cursor[B.cell_off + i] = st;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += incl;
        __syncthreads();
    }
}

static __global__ void k_cell_fill(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    const int pos = atomicAdd(&sh.cell_cursor[cell_of(B, sh.part[p].X)], 1);
    sh.cell_list[pos] = p;
}

// Neighbour list of p: every particle whose centre lies within
// 2R + max(2, lub_cut) (a node owned before the move lies within R + |U| <=
// R + 1 of the new centre, and lubrication acts below a gap of lub_cut).
// One warp per particle; lane k scans cell k of the 3x3x3 block around p.
// FP32 distances against a slightly larger radius give a superset of the
// exact list, which is harmless for both users (claims and pair forces).
// The list is sorted by particle index, so the pair-force sums do not
// depend on the order in which the cells were filled.
constexpr int NLIST_WARPS = 4;
static __global__ void __launch_bounds__(32 * NLIST_WARPS) k_nlist(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    __shared__ int s_ids[NLIST_WARPS][NL_MAX];
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * NLIST_WARPS + wib;
    if (p >= NP) return;  // the whole warp leaves together
    const BoxDev& B = boxes[sh.pbox[p]];
    const PartStateF pf = sh.partf[p];
    const float reach = 2.0f * (float)B.rb + fmaxf(2.0f, (float)B.lub_cut);
    const float lim2 = reach * reach * 1.0001f + 1e-3f;
    const float Lf[3] = {(float)B.nx, (float)B.ny, (float)B.nz};
    // the block of cells around the cell of p (from its FP64 position)
    int c[3], lo[3], nr[3];
    const double* X = sh.part[p].X;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int v = (int)(X[a] / B.cell_len[a]);
        c[a] = v < 0 ? 0 : (v >= B.nc[a] ? B.nc[a] - 1 : v);
        lo[a] = B.nc[a] >= 3 ? c[a] - 1 : 0;
        nr[a] = B.nc[a] >= 3 ? 3 : B.nc[a];
    }
    const int ncell = nr[0] * nr[1] * nr[2];
    int s0 = 0, s1 = 0;
    if (lane < ncell) {
        const int k0 = lane % nr[0], k1 = (lane / nr[0]) % nr[1], k2 = lane / (nr[0] * nr[1]);
        const int cc = B.cell_off + wrapi(lo[0] + k0, B.nc[0]) +
                       B.nc[0] * (wrapi(lo[1] + k1, B.nc[1]) + B.nc[1] * wrapi(lo[2] + k2, B.nc[2]));
        s0 = sh.cell_start[cc];
        s1 = s0 + sh.cell_count[cc];
    }
    auto near = [&](int q) {
        if (q == p) return false;
        const PartStateF qf = sh.partf[q];
        const float dx = mimgf(qf.X[0] - pf.X[0], Lf[0]), dy = mimgf(qf.X[1] - pf.X[1], Lf[1]),
                    dz = mimgf(qf.X[2] - pf.X[2], Lf[2]);
        return dx * dx + dy * dy + dz * dz <= lim2;
    };
    int cnt = 0;
    for (int s = s0; s < s1; s++) cnt += near(sh.cell_list[s]) ? 1 : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    int pos = incl - cnt;
    for (int s = s0; s < s1 && pos < NL_MAX; s++) {
        const int q = sh.cell_list[s];
        if (near(q)) s_ids[wib][pos++] = q;
    }
    __syncwarp();
    const int n = total < NL_MAX ? total : NL_MAX;
    int v = lane < n ? s_ids[wib][lane] : 0x7fffffff;
    // bitonic sort of the 32 lanes, ascending
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int u = __shfl_xor_sync(FULL, v, j);
            const bool up = (lane & k) == 0 || k == 32;
            const bool low = (lane & j) == 0;
            v = (low == up) ? min(v, u) : max(v, u);
        }
    if (lane < n) sh.nlist[(size_t)p * NL_MAX + lane] = v;
    if (lane == 0) {
        sh.nlist_n[p] = n;
        if (total > NL_MAX) set_err(sh.err, ERR_OVERFLOW);
    }
}

// ------------------------------------------------------------- remap
// Warp per particle p: scan the nodes around X_p and record every node whose
// solid/fluid status or owner changes.  A node belongs to the particle whose
// centre is nearest among those within R (|x - X|^2 <= R^2, minimum image);
// ties go to the lower index.  Events: covered (fluid -> p), uncovered
// (p -> fluid), transfer (q -> p, no fluid involved).  Distances are FP32
// (relative to p, from the FP32 particle copy) unless they fall within
// `band` of R^2, where the FP64 value, evaluated without contraction as in a
// plain sequential evaluation, decides.  FP64 is slow on this GPU, so it is
// kept off the common path.
constexpr int DETECT_WARPS = 4;
static __global__ void __launch_bounds__(32 * DETECT_WARPS, 6) k_remap_detect(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    __shared__ float s_rq[DETECT_WARPS][NL_MAX][3];  // X_q - X_p, minimum image
    __shared__ int s_nid[DETECT_WARPS][NL_MAX];
    __shared__ int s_cl[DETECT_WARPS][NL_MAX];  // entries of neighbours within 2R (+ slack)
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * DETECT_WARPS + wib;
    if (p >= NP) return;  // the whole warp leaves together
    const int b = sh.pbox[p];
    const BoxDev& B = boxes[b];
    const PartStateF pf = sh.partf[p];
    // FP32 distances (spheres) or quadratic forms (spheroids) decide away
    // from the surface, the FP64 test (inside_shape) within a band of it
    const bool sph = B.aspect == 1.0;
    const double R = B.rb, R2 = B.radius * B.radius;
    const double L[3] = {(double)B.nx, (double)B.ny, (double)B.nz};
    const float Lf[3] = {(float)B.nx, (float)B.ny, (float)B.nz};
    const int nn = sh.nlist_n[p];
    // A node inside p can also be inside q only if |X_q - X_p| <= 2R (R the
    // bounding radius): those neighbours (the close list; 0.05 of slack
    // covers the FP32 centres) decide the claims of nodes inside p.  A node
    // p owned but left may lie within 2R + 1.5 of q, so that rare case scans
    // the whole list.
    const float rcl = 2.0f * (float)R + 0.05f;
    int ncl = 0;
    {
        bool close = false;
        if (lane < nn) {  // nn <= NL_MAX = 32
            const int q = sh.nlist[(size_t)p * NL_MAX + lane];
            s_nid[wib][lane] = q;
            const PartStateF qf = sh.partf[q];
            float d2 = 0.f;
            for (int a = 0; a < 3; a++) {
                const float v = mimgf(qf.X[a] - pf.X[a], Lf[a]);
                s_rq[wib][lane][a] = v;
                d2 += v * v;
            }
            close = d2 <= rcl * rcl;
        }
        const unsigned cm = __ballot_sync(0xffffffffu, close);
        if (close) s_cl[wib][__popc(cm & ((1u << lane) - 1u))] = lane;
        ncl = __popc(cm);
    }
    __syncwarp();
    // window: every node within R + 1.5 of the centre (a node owned before
    // the move lies within R + |U| <= R + 1 of the new centre; the 0.5 of
    // slack covers the FP32 centre)
    const float reach = (float)R + 1.5f;
    int lo[3], span[3];
    float off[3];  // X_p - lo: node (lo + k) sits at k - off from the centre
    const int dims[3] = {B.nx, B.ny, B.nz};
    for (int a = 0; a < 3; a++) {
        lo[a] = (int)ceilf(pf.X[a] - reach);
        off[a] = pf.X[a] - (float)lo[a];
        span[a] = (int)floorf(pf.X[a] + reach) - lo[a] + 1;
        if (span[a] > dims[a]) span[a] = dims[a];
    }
    const int total = span[0] * span[1] * span[2];
    const float Rf2o = (float)((R + 1.5) * (R + 1.5));
    const float R2f = (float)R2;
    // FP32 positions near L are off by up to about L * 2^-24; the bands below
    // keep every FP32 decision at least twice that error away from the surface
    const double eps_pos = 1.2e-7 * (double)max(B.nx, max(B.ny, B.nz));
    const float band = (float)(0.02 + 2e-3 * R * R + 4.0 * (R + 1.5) * eps_pos);
    const float qlim = (float)(R * R) + band;  // no node beyond this is inside q
    // spheroid prefilter: F = R^2 (d.e)^2 + c^2 (|d|^2 - (d.e)^2) against
    // R^2 c^2 in FP32.  |grad F| <= 2 max(R^2, c^2) |d| within the window, so
    // the position error moves F by at most that times eps_pos; FP32
    // rounding of F adds a few ulps of R^2 c^2; FP64 decides within sband
    const double* Ep = sh.part[p].E;
    const float ex_ = (float)Ep[0], ey_ = (float)Ep[1], ez_ = (float)Ep[2];
    const double cRd = B.aspect * B.radius;
    const float cR = (float)cRd;
    const float R2s = (float)R2, c2s = cR * cR, R2c2 = R2s * c2s;
    const double gmax = 2.0 * fmax(R2, cRd * cRd) * (R + 1.5);
    const float sband = (float)(0.05 + 4.0 * gmax * eps_pos + 1e-6 * R2 * cRd * cRd);
    for (int base = 0; base < total; base += 32) {
        const int idx = base + lane;
        int ev_old = 0, ev_new = 0, node = 0;
        bool have = false;
        if (idx < total) {
            const int kx = idx % span[0], ky = (idx / span[0]) % span[1], kz = idx / (span[0] * span[1]);
            const float fx = mimgf((float)kx - off[0], Lf[0]), fy = mimgf((float)ky - off[1], Lf[1]),
                        fz = mimgf((float)kz - off[2], Lf[2]);
            const float d2f = fx * fx + fy * fy + fz * fz;
            if (d2f <= Rf2o) {
                const int gx = wrapi(lo[0] + kx, B.nx), gy = wrapi(lo[1] + ky, B.ny), gz = wrapi(lo[2] + kz, B.nz);
                // FP64 inside test of this node for particle q; d2 = squared
                // centre distance (the claim goes to the nearest centre)
                auto exact_in = [&](int q, double& d2) {
                    const double* C = sh.part[q].X;
                    const double dx = mimg((double)gx - C[0], L[0]), dy = mimg((double)gy - C[1], L[1]),
                                 dz = mimg((double)gz - C[2], L[2]);
                    d2 = dist2_nc(dx, dy, dz);
                    return inside_shape(B, dx, dy, dz, sh.part[q].E);
                };
                const int n = gx + B.nx * (gy + B.ny * gz);
                const int own = __ldg(B.owner + n);
                if (own != OWN_WALL) {
                    double d2p = -1.0;
                    bool inside;
                    if (sph) {
                        if (fabsf(d2f - R2f) > band) inside = d2f < R2f;
                        else inside = exact_in(p, d2p);
                    } else {
                        const float sf = fx * ex_ + fy * ey_ + fz * ez_;
                        const float Ff = R2s * sf * sf + c2s * (d2f - sf * sf);
                        if (fabsf(Ff - R2c2) > sband) inside = Ff < R2c2;
                        else inside = exact_in(p, d2p);
                    }
                    if (inside || own == p) {
                        bool other = false, anyone = false;
                        const int nk = inside ? ncl : nn;
                        for (int kk = 0; kk < nk; kk++) {
                            const int k = inside ? s_cl[wib][kk] : kk;
                            const float ex = mimgf(fx - s_rq[wib][k][0], Lf[0]);
                            const float ey = mimgf(fy - s_rq[wib][k][1], Lf[1]);
                            const float ez = mimgf(fz - s_rq[wib][k][2], Lf[2]);
                            if (ex * ex + ey * ey + ez * ez > qlim) continue;
                            const int q = s_nid[wib][k];
                            double d2q;
                            if (exact_in(q, d2q)) {
                                anyone = true;
                                if (inside) {
                                    if (d2p < 0.0) exact_in(p, d2p);
                                    if (d2q < d2p || (d2q == d2p && q < p)) other = true;
                                }
                            }
                        }
                        const bool claim = inside && !other;
                        if (claim && own != p) {
                            have = true;
                            ev_old = own;
                            ev_new = p;
                        } else if (!claim && own == p && !anyone) {
                            have = true;
                            ev_old = p;
                            ev_new = OWN_FLUID;
                        }
                        node = n;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, have);
        if (m) {
            int basepos = 0;
            if (lane == 0) basepos = atomicAdd(sh.ev_count, __popc(m));
            basepos = __shfl_sync(0xffffffffu, basepos, 0);
            if (have) {
                const int pos = basepos + __popc(m & ((1u << lane) - 1u));
                if (pos < sh.ev_cap) sh.events[pos] = make_int4(node, b, ev_old, ev_new);
                else set_err(sh.err, ERR_OVERFLOW);
            }
        }
    }
}

__device__ __forceinline__ int ev_total(const Shared& sh) {
    const int c = *sh.ev_count;
    return c < sh.ev_cap ? c : sh.ev_cap;
}

// new status of every event node; the old owner is kept in evmark (+3)
static __global__ void k_remap_mark(const BoxDev* __restrict__ boxes, Shared sh) {
    const int cnt = ev_total(sh);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const int4 ev = sh.events[e];
        const BoxDev& B = boxes[ev.y];
        B.evmark[ev.x] = ev.z + 3;
        B.owner[ev.x] = ev.w;
        B.flags[ev.x] = ev.w != OWN_FLUID ? FL_SOLID : 0;
    }
}

__device__ __forceinline__ int nbr_index(const BoxDev& B, int n, int dx, int dy, int dz) {
    const int x = n % B.nx, y = (n / B.nx) % B.ny, z = n / (B.nx * B.ny);
    return wrapi(x + dx, B.nx) + B.nx * (wrapi(y + dy, B.ny) + B.ny * wrapi(z + dz, B.nz));
}
__device__ __forceinline__ bool old_solid(const BoxDev& B, int n) {
    const int m = B.evmark[n];
    if (m) return (m - 3) != OWN_FLUID;
    return B.flags[n] & FL_SOLID;
}
// refill of an uncovered node (Eqs. eqn_rho_neu and masscorr): mean density
// of the neighbours that were fluid, times the mass-correction factor; the
// surface velocity of the particle that left it.
template <class R>
struct Refill {
    R rho[2];
    R us[3];
    double r[3];
};
template <class R>
__device__ Refill<R> refill_of(const BoxDev& B, const Shared& sh, int n, int q, const R* rcur, int mslot_cur) {
    Refill<R> o;
    double corr[2] = {1.0, 1.0};
    if (B.c0 != 0.0) {
        const double rsum = B.rho_init[0] + B.rho_init[1];
        for (int c = 0; c < 2; c++)
            corr[c] = 1.0 - B.c0 * (rsum / B.rho_init[c]) * (B.mass_acc[mslot_cur * 2 + c] - B.mass0[c]) / (double)B.N;
    }
    for (int c = 0; c < 2; c++) {
        R sum = R(0);
        int cnt = 0;
#pragma unroll
        for (int i = 1; i < 19; i++) {
            const int m = nbr_index(B, n, cx(i), cy(i), cz(i));
            if (!old_solid(B, m)) {
                sum += rcur[2 * (size_t)m + c];
                cnt++;
            }
        }
        const R rbar = cnt ? sum / (R)cnt : (R)B.rho_init[c];
        o.rho[c] = (R)((double)rbar * corr[c]);
    }
    const int x = n % B.nx, y = (n / B.nx) % B.ny, z = n / (B.nx * B.ny);
    const PartState ps = sh.part[q];
    o.r[0] = mimg((double)x - ps.X[0], B.nx);
    o.r[1] = mimg((double)y - ps.X[1], B.ny);
    o.r[2] = mimg((double)z - ps.X[2], B.nz);
    o.us[0] = (R)(ps.U[0] + ps.W[1] * o.r[2] - ps.W[2] * o.r[1]);
    o.us[1] = (R)(ps.U[1] + ps.W[2] * o.r[0] - ps.W[0] * o.r[2]);
    o.us[2] = (R)(ps.U[2] + ps.W[0] * o.r[1] - ps.W[1] * o.r[0]);
    return o;
}

__device__ __forceinline__ void add_force_torque(const Shared& sh, int p, const double r[3], const double F[3]) {
    double t[3];
    cross3(r, F, t);
    for (int a = 0; a < 3; a++) {
        atomicAdd(&sh.force[(size_t)p * 6 + a], F[a]);
        atomicAdd(&sh.force[(size_t)p * 6 + 3 + a], t[a]);
    }
}

__device__ __forceinline__ void node_rel(const BoxDev& B, const Shared& sh, int n, int p, double r[3]) {
    const int x = n % B.nx, y = (n / B.nx) % B.ny, z = n / (B.nx * B.ny);
    const PartState& ps = sh.part[p];
    r[0] = mimg((double)x - ps.X[0], B.nx);
    r[1] = mimg((double)y - ps.X[1], B.ny);
    r[2] = mimg((double)z - ps.X[2], B.nz);
}

// Cover / uncover.  PAR is the parity of the coming fused step.  Before an
// even step f_i of a node sits in its own slot i; before an odd step it sits
// in slot opp(i) of the neighbour x - c_i, whatever that neighbour's status
// (the even step stores a population reflected at a solid node in that
// node's slot).  So a status change moves nothing: a covered node gives the
// momentum of its populations to the particle, an uncovered node gets
// f^eq(rho_new, u_s) in the same places, and the particle loses the
// momentum of the created fluid.
template <class P, int PAR>
static __global__ void k_remap_apply(const BoxDev* __restrict__ boxes, Shared sh, int rc, int mslot_cur) {
    using R = typename P::real;
    const int cnt = ev_total(sh);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const int4 ev = sh.events[e];
        const int w = ev.x, old = ev.z, nw = ev.w;
        if (old != OWN_FLUID && nw != OWN_FLUID) continue;  // transfer between particles
        const BoxDev& B = boxes[ev.y];
        const Pop<P> pop(B);
        const R* rcur = reinterpret_cast<const R*>(B.rho[rc]);
        const bool covered = (old == OWN_FLUID);
        // node holding f_i of w before the coming step
        auto src = [&](int i) { return PAR == 0 ? w : nbr_index(B, w, -cx(i), -cy(i), -cz(i)); };
        auto slot = [&](int i) { return PAR == 0 ? i : opp(i); };
        if (covered) {
            atomicAdd(&sh.counters[ev.y * 2 + 0], 1ull);
            double mom_w[3] = {0, 0, 0};
            for (int c = 0; c < 2; c++) {
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    const R v = pop.load(c, slot(i), src(i));
                    mom_w[0] += (double)v * cx(i);
                    mom_w[1] += (double)v * cy(i);
                    mom_w[2] += (double)v * cz(i);
                }
            }
            double r[3];
            node_rel(B, sh, w, nw, r);
            add_force_torque(sh, nw, r, mom_w);
        } else {
            const Refill<R> rf = refill_of<R>(B, sh, w, old, rcur, mslot_cur);
            sh.ev_rho[(size_t)e * 2 + 0] = (double)rf.rho[0];
            sh.ev_rho[(size_t)e * 2 + 1] = (double)rf.rho[1];
            atomicAdd(&sh.counters[ev.y * 2 + 1], 1ull);
            // the 18 moving populations; the density rho_new (set by
            // k_remap_finish) makes the rest population rho_new minus them
            for (int c = 0; c < 2; c++) {
#pragma unroll
                for (int i = 1; i < 19; i++)
                    pop.store(c, slot(i), src(i), feq_rt<R>(i, rf.rho[c], rf.us[0], rf.us[1], rf.us[2]));
            }
            // the particle loses the momentum of the created fluid
            // (Eq. eqn_ladd_vernichtenunderzeugen, sign from conservation)
            const double rs = (double)rf.rho[0] + (double)rf.rho[1];
            const double F[3] = {-rs * (double)rf.us[0], -rs * (double)rf.us[1], -rs * (double)rf.us[2]};
            add_force_torque(sh, old, rf.r, F);
        }
    }
}

__device__ __forceinline__ void shell_update(const BoxDev& B, int n) {
    const uint8_t f = B.flags[n];
    if (!(f & FL_SOLID)) return;
    bool shl = false;
#pragma unroll
    for (int i = 1; i < 19; i++)
        if (!(B.flags[nbr_index(B, n, cx(i), cy(i), cz(i))] & FL_SOLID)) shl = true;
    B.flags[n] = FL_SOLID | (shl ? FL_SHELL : 0);
}

template <class R>
static __global__ void k_remap_finish(const BoxDev* __restrict__ boxes, Shared sh, int rc) {
    const int cnt = ev_total(sh);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const int4 ev = sh.events[e];
        const BoxDev& B = boxes[ev.y];
        const int w = ev.x;
        R* rcur = reinterpret_cast<R*>(B.rho[rc]);
        if (ev.z == OWN_FLUID) {
            rcur[2 * (size_t)w] = R(0);
            rcur[2 * (size_t)w + 1] = R(0);
        } else if (ev.w == OWN_FLUID) {
            rcur[2 * (size_t)w] = (R)sh.ev_rho[(size_t)e * 2 + 0];
            rcur[2 * (size_t)w + 1] = (R)sh.ev_rho[(size_t)e * 2 + 1];
        }
        B.evmark[w] = 0;
        // the particles whose shell lists this event can change: the old and
        // new owner of w and the owners of its solid neighbours (their
        // fluid-neighbour masks)
        if (ev.z >= 0) sh.shell_dirty[ev.z] = 1;
        if (ev.w >= 0) sh.shell_dirty[ev.w] = 1;
#pragma unroll
        for (int i = 1; i < 19; i++) {
            const int o = B.owner[nbr_index(B, w, cx(i), cy(i), cz(i))];
            if (o >= 0) sh.shell_dirty[o] = 1;
        }
        // A solid node left without fluid neighbours takes density 0: the
        // fused step may have counted reflected populations in it while it
        // was a shell node, and no later pass rewrites it (the particle's
        // Shan-Chen force reads it through its shell neighbours).
        auto update = [&](int n) {
            shell_update(B, n);
            if (B.flags[n] == FL_SOLID) {
                rcur[2 * (size_t)n] = R(0);
                rcur[2 * (size_t)n + 1] = R(0);
            }
        };
        update(w);
#pragma unroll
        for (int i = 1; i < 19; i++) update(nbr_index(B, w, cx(i), cy(i), cz(i)));
    }
}

// ------------------------------------------------------- virtual fluid
// Shell nodes get the mean density of their fluid neighbours plus the
// particle colour on red (Delta rho > 0) or blue (Delta rho < 0) (Sec. IV).
template <class R>
static __global__ void __launch_bounds__(128, 8) k_shell_density(const BoxDev* __restrict__ boxes, Shared sh, int rc, int NP) {
    __shared__ int s_q[4][64];
    __shared__ int s_qc[4][64];  // x | y << 16 of the queued node
    __shared__ int s_qz[4][64];  // z of the queued node
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * 4 + wib;
    if (p >= NP) return;  // the whole warp leaves together
    const BoxDev& B = boxes[sh.pbox[p]];
    const PartStateF pf = sh.partf[p];
    R* __restrict__ rcur = reinterpret_cast<R*>(B.rho[rc]);
    const uint8_t* __restrict__ flags = B.flags;
    const int32_t* __restrict__ owner = B.owner;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const size_t N = (size_t)B.N;
    const float R_ = (float)B.rb;  // bounding radius (the radius for spheres)
    const R col = (R)sh.color[p];
    // window: every node within R + 0.5 of the centre (the shell nodes of p
    // lie within R; the 0.5 of slack covers the FP32 centre)
    const float reach = R_ + 0.5f;
    int lo[3], span[3];
    float off[3];  // X - lo: node (lo + k) sits at k - off from the centre
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++) {
        lo[a] = (int)ceilf(pf.X[a] - reach);
        off[a] = pf.X[a] - (float)lo[a];
        span[a] = (int)floorf(pf.X[a] + reach) - lo[a] + 1;
        if (span[a] > dims[a]) span[a] = dims[a];
    }
    const int total = span[0] * span[1] * span[2];
    const int scap = sh.shell_cap;
    int4* __restrict__ slist = sh.shell_list + (size_t)p * scap;
    if (!sh.shell_dirty[p]) {
        // No event near p since its list was built: the shell nodes and
        // their fluid-neighbour masks are unchanged, only the densities are
        // new (the whole warp takes this branch together).
        const int ns = sh.shell_n[p];
        const int nxy = nx * ny;
        for (int k = lane; k < ns; k += 32) {
            const int4 e = slist[k];
            const int n = e.x;
            const unsigned fmask = (unsigned)e.y;
            const int gx = e.z & 0xffff, gy = (int)((unsigned)e.z >> 16), gz = e.w;
            const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
            const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
            const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
            R s0 = R(0), s1 = R(0);
#pragma unroll
            for (int i = 1; i < 19; i++) {
                if (!((fmask >> i) & 1u)) continue;
                const int m = n + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) +
                              (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) + (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
                s0 += rcur[2 * (size_t)m];
                s1 += rcur[2 * (size_t)m + 1];
            }
            const R cnt = (R)__popc(fmask);
            R r0 = s0 / cnt, r1 = s1 / cnt;
            if (col > R(0)) r0 += col;
            else if (col < R(0)) r1 -= col;
            rcur[2 * (size_t)n] = r0;
            rcur[2 * (size_t)n + 1] = r1;
        }
        return;
    }
    // virtual density of one shell node n of p, and its entry k of p's
    // shell list (node, mask of fluid neighbours, coordinates)
    const int nxy = nx * ny;
    auto process = [&](int n, int gx, int gy, int gz, int k) {
        // wrap-aware offsets to the neighbours along each axis
        const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
        const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
        const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
        R s0 = R(0), s1 = R(0);
        int cnt = 0;
        unsigned fmask = 0;  // bit i: n + c_i is fluid (a link)
#pragma unroll
        for (int i = 1; i < 19; i++) {
            const int m = n + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) + (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) +
                          (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
            if (!(flags[m] & FL_SOLID)) {
                s0 += rcur[2 * (size_t)m];
                s1 += rcur[2 * (size_t)m + 1];
                cnt++;
                fmask |= 1u << i;
            }
        }
        if (k < scap) slist[k] = make_int4(n, (int)fmask, (int)((unsigned)gx | ((unsigned)gy << 16)), gz);
        R r0 = s0 / (R)cnt, r1 = s1 / (R)cnt;
        if (col > R(0)) r0 += col;
        else if (col < R(0)) r1 -= col;
        rcur[2 * (size_t)n] = r0;
        rcur[2 * (size_t)n + 1] = r1;
    };
    // FP32 prefilter only (every shell node of p lies within R); the shell
    // flag and the owner decide.  No FP64 here: it is slow on this GPU.
    // Shell nodes are queued as they are found and handled 32 at a time;
    // they are also listed for k_couple.
    const float lim = (R_ + 0.5f) * (R_ + 0.5f);
    int nq = 0, done = 0;  // warp-uniform: queue length (< 64), nodes handled
    for (int base = 0;; base += 32) {
        const int idx = base + lane;
        bool take = false;
        int n = 0, gx = 0, gy = 0, gz = 0;
        if (idx < total) {
            const int kx = idx % span[0], ky = (idx / span[0]) % span[1], kz = idx / (span[0] * span[1]);
            const float dx = mimgf((float)kx - off[0], (float)nx), dy = mimgf((float)ky - off[1], (float)ny),
                        dz = mimgf((float)kz - off[2], (float)nz);
            if (dx * dx + dy * dy + dz * dz <= lim) {
                gx = wrapi(lo[0] + kx, nx);
                gy = wrapi(lo[1] + ky, ny);
                gz = wrapi(lo[2] + kz, nz);
                n = gx + nx * (gy + ny * gz);
                take = (__ldg(flags + n) & FL_SHELL) && __ldg(owner + n) == p;
            }
        }
        const unsigned m = __ballot_sync(FULL, take);
        if (take) {
            const int pos = nq + __popc(m & ((1u << lane) - 1u));
            s_q[wib][pos] = n;
            s_qc[wib][pos] = (int)((unsigned)gx | ((unsigned)gy << 16));
            s_qz[wib][pos] = gz;
        }
        nq += __popc(m);
        __syncwarp();
        const bool last = base + 32 >= total;  // the final round drains the queue
        if (nq >= 32 || (last && nq > 0)) {
            const int k = nq < 32 ? nq : 32;
            const int item = lane < k ? s_q[wib][nq - k + lane] : -1;
            const int ic = lane < k ? s_qc[wib][nq - k + lane] : 0;
            const int iz = lane < k ? s_qz[wib][nq - k + lane] : 0;
            __syncwarp();
            nq -= k;
            if (item >= 0) process(item, ic & 0xffff, (int)((unsigned)ic >> 16), iz, done + lane);
            done += k;
        }
        if (last && nq == 0) break;
    }
    if (lane == 0) {
        sh.shell_n[p] = done < scap ? done : scap;
        if (done > scap) set_err(sh.err, ERR_OVERFLOW);
        else sh.shell_dirty[p] = 0;
    }
}

// ----------------------------------------------------- fluid -> particle
// Coupling terms of each particle that live on its surface, after the fused
// step; one block per particle over its shell nodes s (solid nodes of p with
// a fluid D3Q19 neighbour, listed by k_shell_density in this step):
//   * the Shan-Chen force of the virtual fluid at s on the particle
//     (Eq. eqn_shan_chen_particle): F = sum_c -g Psi^c(s) sum_i W_i
//     Psi^cbar(s + c_i) c_i, torque (s - X) x F;
//   * every link from a fluid neighbour x = s + c_i to s, direction
//     j = opp(i).  The post-collision f*_j of x belongs, reflected, in slot
//     j of s (even step) or slot i of x (odd step).  With reflect = 1 the
//     fused step stored it there; with reflect = 0 it stored it as if s were
//     fluid (slot i of x after an even step, slot j of s after an odd one)
//     and counted it in the density of s, and this kernel moves it.  The
//     value gets the moving-wall term, b = f*_j - 6 zeta_j rho^c(x)
//     (u_s . c_j) with u_s =
//     U + omega x r at the link midpoint r = x + c_j / 2 - X
//     (Eq. eqn_ladd_bewegtewand), and the particle receives
//     (2 f*_j - 6 zeta_j rho^c(x) u_s . c_j) c_j with torque r x F
//     (Eq. eqn_bounce-back-force).  rho(t+1) at x gets the change of the
//     value (reflect = 1) or all of it (reflect = 0), and the fluid mass the
//     step produced gets the change.  In deviation storage the density
//     field takes the exact change b - f*_j: the rounding of the re-encoded
//     value lands in the rest population of x, which is rho^c minus the 18
//     stored ones; an unchanged value (no wall term) moves bit for bit.
// A link belongs to the owner of its solid end, so each slot is written
// once; the density updates are atomic because several links can share a
// fluid node.  Static walls (owner -2) reflect without a wall
// term and need nothing here.  rho^c(x) is the density field of the current
// step (the fused step's moments up to rounding order).
constexpr int COUPLE_THREADS = 256;
template <class P>
static __global__ void __launch_bounds__(COUPLE_THREADS)
    k_couple(const BoxDev* __restrict__ boxes, Shared sh, int rc, int rn, int mslot, int par, int reflect) {
    using R = typename P::real;
    using S = typename P::st;
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ R s_red[COUPLE_THREADS / 32][8];
    const int p = blockIdx.x;
    const BoxDev& B = boxes[sh.pbox[p]];
    const Pop<P> pop(B);
    const auto& ps = part_ptr<R>(sh)[p];
    const size_t N = (size_t)B.N;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    using R2 = typename Real2<R>::type;
    using S2 = typename P::st2;
    const R2* __restrict__ rcur2 = rpair<R>(B.rho[rc]);
    R2* __restrict__ rnext2 = rpair<R>(B.rho[rn]);
    double* __restrict__ mass_acc = B.mass_acc;
    const R rho0 = (R)B.rho0, irho0 = R(1) / (R)B.rho0, g = (R)B.g;
    const R wax = (R)B.scw_axis, wdg = (R)B.scw_diag;
    const R Lx = (R)nx, Ly = (R)ny, Lz = (R)nz;
    const R X0 = (R)ps.X[0], X1 = (R)ps.X[1], X2 = (R)ps.X[2];
    const R U0 = (R)ps.U[0], U1 = (R)ps.U[1], U2 = (R)ps.U[2];
    const R W0 = (R)ps.W[0], W1 = (R)ps.W[1], W2 = (R)ps.W[2];
    R acc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R dm0 = R(0), dm1 = R(0);
    // the shell nodes found by k_shell_density in this step
    const int ns = sh.shell_n[p];
    const int4* __restrict__ list = sh.shell_list + (size_t)p * sh.shell_cap;
    // (1) links: one item per (direction i, shell node s), direction-major,
    // so that neighbouring threads touch neighbouring nodes of one array.
    // Each thread takes U items at a time and issues all their loads before
    // any store, so that U independent chains are in flight.
    constexpr int U = 4;
    const int nitems = 18 * ns;
    for (int k0 = threadIdx.x; k0 < nitems; k0 += U * COUPLE_THREADS) {
        int iu[U], mu[U];
        S2* pu[U];
        ptrdiff_t mv[U];  // pairs from the slot read to the slot written
        S2 rawu[U];
        R2 rru[U];
        int4 eu[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = k0 + u * COUPLE_THREADS;
            ok[u] = k < nitems;
            iu[u] = 1;
            if (ok[u]) {
                iu[u] = 1 + k / ns;
                eu[u] = list[k - (iu[u] - 1) * ns];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int i = iu[u];
            ok[u] = ok[u] && ((eu[u].y >> i) & 1);  // s + c_i fluid: a link
            mu[u] = 0;
            mv[u] = 0;
            pu[u] = nullptr;
            if (ok[u]) {
                const int s = eu[u].x;
                const int gx = eu[u].z & 0xffff, gy = (int)((unsigned)eu[u].z >> 16), gz = eu[u].w;
                const int m = wrap1(gx + kC[i][0], nx) + nx * (wrap1(gy + kC[i][1], ny) + ny * wrap1(gz + kC[i][2], nz));
                mu[u] = m;
                // the reflected pair f*_j belongs after an even step in slot
                // j = opp(i) of s, after an odd step in slot opp(j) = i of
                // m; unreflected it sits in the other of the two
                const bool at_s = (par == 0) == (reflect != 0);
                pu[u] = at_s ? pop.pair(opp(i), s) : pop.pair(i, m);
                if (!reflect) mv[u] = at_s ? pop.pair(i, m) - pu[u] : pop.pair(opp(i), s) - pu[u];
                rawu[u] = *pu[u];
                rru[u] = __ldg(rcur2 + m);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (!ok[u]) continue;
            const int i = iu[u], m = mu[u];
            const int ix = kC[i][0], iy = kC[i][1], iz = kC[i][2];
            const int gx = eu[u].z & 0xffff, gy = (int)((unsigned)eu[u].z >> 16), gz = eu[u].w;
            // link from the fluid node m to s; c_j = -c_i; midpoint s + c_i / 2
            const R r0 = mimg_r<R>((R)gx - X0, Lx) + R(0.5) * (R)ix;
            const R r1 = mimg_r<R>((R)gy - X1, Ly) + R(0.5) * (R)iy;
            const R r2 = mimg_r<R>((R)gz - X2, Lz) + R(0.5) * (R)iz;
            const R us0 = U0 + W1 * r2 - W2 * r1, us1 = U1 + W2 * r0 - W0 * r2, us2 = U2 + W0 * r1 - W1 * r0;
            const R cu6 = -R(6) * (i <= 6 ? wgt<R>(1) : wgt<R>(7)) * (us0 * (R)ix + us1 * (R)iy + us2 * (R)iz);
            const S2 raw = rawu[u];
            R fs[2], wall[2], dr[2] = {R(0), R(0)};
            if constexpr (P::dev) {
                fs[0] = pop.dev_to_f(0, i, raw.x);
                fs[1] = pop.dev_to_f(1, i, raw.y);
            } else {
                fs[0] = raw.x;
                fs[1] = raw.y;
            }
            wall[0] = cu6 * rru[u].x;
            wall[1] = cu6 * rru[u].y;
            if (cu6 != R(0) || !reflect) {
                S2 q = raw;
                if constexpr (P::dev) {
                    // a value without a wall term moves bit for bit; the
                    // density field takes the exact change b - f* of a
                    // re-encoded one (its rounding lands in the rest
                    // population, which is rho minus the 18 stored values)
                    if (wall[0] != R(0)) {
                        q.x = pop.f_to_dev(0, i, fs[0] - wall[0]);
                        dr[0] = -wall[0];
                    }
                    if (wall[1] != R(0)) {
                        q.y = pop.f_to_dev(1, i, fs[1] - wall[1]);
                        dr[1] = -wall[1];
                    }
                } else {
                    q.x = fs[0] - wall[0];
                    q.y = fs[1] - wall[1];
                    dr[0] = q.x - fs[0];
                    dr[1] = q.y - fs[1];
                }
                pu[u][mv[u]] = q;
                red_add2<R>(rnext2 + m, reflect ? dr[0] : dr[0] + fs[0], reflect ? dr[1] : dr[1] + fs[1]);
                dm0 += dr[0];
                dm1 += dr[1];
            }
            const R mag = (R(2) * fs[0] - wall[0]) + (R(2) * fs[1] - wall[1]);
            const R F0 = -mag * (R)ix, F1 = -mag * (R)iy, F2 = -mag * (R)iz;
            acc[0] += F0;
            acc[1] += F1;
            acc[2] += F2;
            acc[3] += r1 * F2 - r2 * F1;
            acc[4] += r2 * F0 - r0 * F2;
            acc[5] += r0 * F1 - r1 * F0;
        }
    }
    // (2) the Shan-Chen force of the virtual fluid at each shell node
    for (int k = threadIdx.x; k < ns; k += COUPLE_THREADS) {
        const int4 e = list[k];
        const int s = e.x;
        const int gx = e.z & 0xffff, gy = (int)((unsigned)e.z >> 16), gz = e.w;
        R sr0 = R(0), sr1 = R(0), sr2 = R(0), sb0 = R(0), sb1 = R(0), sb2 = R(0);
#pragma unroll
        for (int i = 1; i < 19; i++) {
            const int m = wrap1(gx + cx(i), nx) + nx * (wrap1(gy + cy(i), ny) + ny * wrap1(gz + cz(i), nz));
            const R w = is_axis(i) ? wax : wdg;
            const R2 rm = __ldg(rcur2 + m);
            const R pr = w * psi_of<R>(rm.x, rho0, irho0);
            const R pb = w * psi_of<R>(rm.y, rho0, irho0);
            sr0 += pr * (R)cx(i);
            sr1 += pr * (R)cy(i);
            sr2 += pr * (R)cz(i);
            sb0 += pb * (R)cx(i);
            sb1 += pb * (R)cy(i);
            sb2 += pb * (R)cz(i);
        }
        const R rs0 = mimg_r<R>((R)gx - X0, Lx), rs1 = mimg_r<R>((R)gy - X1, Ly), rs2 = mimg_r<R>((R)gz - X2, Lz);
        const R2 rs = __ldg(rcur2 + s);
        const R psr = psi_of<R>(rs.x, rho0, irho0), psb = psi_of<R>(rs.y, rho0, irho0);
        const R F0 = -g * (psr * sb0 + psb * sr0), F1 = -g * (psr * sb1 + psb * sr1), F2 = -g * (psr * sb2 + psb * sr2);
        acc[0] += F0;
        acc[1] += F1;
        acc[2] += F2;
        acc[3] += rs1 * F2 - rs2 * F1;
        acc[4] += rs2 * F0 - rs0 * F2;
        acc[5] += rs0 * F1 - rs1 * F0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 6; a++) acc[a] += __shfl_xor_sync(FULL, acc[a], o);
        dm0 += __shfl_xor_sync(FULL, dm0, o);
        dm1 += __shfl_xor_sync(FULL, dm1, o);
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 6; a++) s_red[wib][a] = acc[a];
        s_red[wib][6] = dm0;
        s_red[wib][7] = dm1;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int a = threadIdx.x;
        R v = s_red[0][a];
#pragma unroll
        for (int w = 1; w < COUPLE_THREADS / 32; w++) v += s_red[w][a];
        // the only writer of this particle's accumulator in this kernel
        if (a < 6) sh.force[(size_t)p * 6 + a] += (double)v;
        else if (v != R(0)) atomicAdd(&mass_acc[mslot * 2 + (a - 6)], (double)v);
    }
}

// shell nodes of static walls (colour 0); only boxes that have walls
template <class R>
static __global__ void k_wall_shell(const BoxDev* __restrict__ boxes, int b, int rc) {
    const BoxDev& B = boxes[b];
    R* rcur = reinterpret_cast<R*>(B.rho[rc]);
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < B.N; n += gridDim.x * blockDim.x) {
        if (B.owner[n] != OWN_WALL || !(B.flags[n] & FL_SHELL)) continue;
        R s0 = R(0), s1 = R(0);
        int cnt = 0;
        for (int i = 1; i < 19; i++) {
            const int m = nbr_index(B, n, cx(i), cy(i), cz(i));
            if (!(B.flags[m] & FL_SOLID)) {
                s0 += rcur[2 * (size_t)m];
                s1 += rcur[2 * (size_t)m + 1];
                cnt++;
            }
        }
        rcur[2 * (size_t)n] = s0 / (R)cnt;
        rcur[2 * (size_t)n + 1] = s1 / (R)cnt;
    }
}

// --------------------------------------------------------------- MD
// Pair force on p from q, r = X_p - X_q (minimum image):
//   Hertz (Eq. eq:hertz): -dV/dr = 5/2 K (2R - r)^{3/2} along r_hat, r < 2R;
//   lubrication (Eq. eqn_ladd_lubrikation): -6 pi nu R^4/(2R)^2 r_hat
//   [r_hat.(U_p - U_q)] (1/h - 1/h_c) for gap h < h_c, h clamped at h_min.
// Spheroids: 2R becomes the contact distance along r_hat (contact_distance)
// and R half of it.
__device__ __forceinline__ void pair_force(const BoxDev& B, const PartState& a, const PartState& b, double F[3]) {
    double r[3] = {mimg(a.X[0] - b.X[0], B.nx), mimg(a.X[1] - b.X[1], B.ny), mimg(a.X[2] - b.X[2], B.nz)};
    const double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (d <= 0.0) return;
    const double rh[3] = {r[0] / d, r[1] / d, r[2] / d};
    const double sigma = contact_distance(B, rh, a.E, b.E), R = 0.5 * sigma;
    if (d < 2.0 * R) {
        const double ov = 2.0 * R - d;
        const double mag = 2.5 * B.k_hertz * ov * sqrt(ov);
        for (int k = 0; k < 3; k++) F[k] += mag * rh[k];
    }
    const double h = d - 2.0 * R;
    if (h < B.lub_cut) {
        const double he = h < B.lub_min ? B.lub_min : h;
        const double du = rh[0] * (a.U[0] - b.U[0]) + rh[1] * (a.U[1] - b.U[1]) + rh[2] * (a.U[2] - b.U[2]);
        const double mag = -6.0 * M_PI * B.nu * R * R * R * R / (4.0 * R * R) * du * (1.0 / he - 1.0 / B.lub_cut);
        for (int k = 0; k < 3; k++) F[k] += mag * rh[k];
    }
}

// FP32 copy of particles [p0, p0 + n) for the FP32 fluid kernels
static __global__ void k_part_to_float(Shared sh, int p0, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const PartState ps = sh.part[p0 + k];
    PartStateF pf;
    for (int a = 0; a < 3; a++) {
        pf.X[a] = (float)ps.X[a];
        pf.U[a] = (float)ps.U[a];
        pf.W[a] = (float)ps.W[a];
    }
    sh.partf[p0 + k] = pf;
}

// coupling forces of the step are saved, then the pair forces are added
// Pair forces (Hertz contact and lubrication) on p, added to the fluid
// force; the fluid part is kept in force_last first.  One warp per particle,
// lane k takes the k-th entry of the (sorted) neighbour list; a fixed
// butterfly sums the lanes, so the result does not depend on timing.
constexpr int MD_WARPS = 4;
static __global__ void __launch_bounds__(32 * MD_WARPS) k_md_forces(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * MD_WARPS + wib;
    if (p >= NP) return;  // the whole warp leaves together
    const BoxDev& B = boxes[sh.pbox[p]];
    double* fp = &sh.force[(size_t)p * 6];
    const double mine = lane < 6 ? fp[lane] : 0.0;
    if (lane < 6) sh.force_last[(size_t)p * 6 + lane] = mine;
    double F[3] = {0.0, 0.0, 0.0};
    const int nn = sh.nlist_n[p];
    if (lane < nn) pair_force(B, sh.part[p], sh.part[sh.nlist[(size_t)p * NL_MAX + lane]], F);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; a++) F[a] += __shfl_xor_sync(FULL, F[a], off);
    if (lane < 3) fp[lane] = mine + F[lane];
}

// Rotation of a spheroid with torque T: L = I(e) omega, L += T, the axis
// turns about L by |L| / I_perp (exact for torque-free motion: de/dt =
// (L x e) / I_perp), then omega = I(e_new)^-1 L; I(e) = I_perp (1 - e e) +
// I_par e e.
__device__ __forceinline__ void rotate_spheroid(const BoxDev& B, double W[3], double e[3], const double T[3]) {
    auto inertia = [&](const double* v, double* o, bool inv) {
        const double a = inv ? 1.0 / B.iperp : B.iperp, b = inv ? 1.0 / B.ipar : B.ipar;
        const double t = e[0] * v[0] + e[1] * v[1] + e[2] * v[2];
        for (int k = 0; k < 3; k++) o[k] = a * v[k] + (b - a) * t * e[k];
    };
    double L[3];
    inertia(W, L, false);
    for (int a = 0; a < 3; a++) L[a] += T[a];
    const double Lm = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    if (Lm > 0.0) {
        const double k[3] = {L[0] / Lm, L[1] / Lm, L[2] / Lm};
        const double th = Lm / B.iperp;
        const double kxe[3] = {k[1] * e[2] - k[2] * e[1], k[2] * e[0] - k[0] * e[2], k[0] * e[1] - k[1] * e[0]};
        const double ct = cos(th), st = sin(th), ke = k[0] * e[0] + k[1] * e[1] + k[2] * e[2];
        double en[3];
        for (int a = 0; a < 3; a++) en[a] = e[a] * ct + kxe[a] * st + k[a] * ke * (1.0 - ct);
        const double nn = sqrt(en[0] * en[0] + en[1] * en[1] + en[2] * en[2]);
        for (int a = 0; a < 3; a++) e[a] = en[a] / nn;
    }
    inertia(L, W, true);
}

// leap-frog: U += F/m, omega += T/J (spheroids: rotate_spheroid), X += U
// (periodic); accumulators zeroed
static __global__ void k_md_integrate(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    double* fp = &sh.force[(size_t)p * 6];
    PartState ps = sh.part[p];
    if (!B.fixed) {
        const double L[3] = {(double)B.nx, (double)B.ny, (double)B.nz};
        if (B.aspect != 1.0) rotate_spheroid(B, ps.W, ps.E, fp + 3);
        for (int a = 0; a < 3; a++) {
            ps.U[a] += fp[a] / B.mass;
            if (B.aspect == 1.0) ps.W[a] += fp[3 + a] / B.inertia;
            double xn = ps.X[a] + ps.U[a];
            xn -= L[a] * floor(xn / L[a]);
            if (xn >= L[a]) xn -= L[a];
            ps.X[a] = xn;
        }
        if (!(ps.U[0] * ps.U[0] + ps.U[1] * ps.U[1] + ps.U[2] * ps.U[2] < 1.0)) set_err(sh.err, ERR_FAST_PARTICLE);
        sh.part[p] = ps;
        PartStateF pf;
        for (int a = 0; a < 3; a++) {
            pf.X[a] = (float)ps.X[a];
            pf.U[a] = (float)ps.U[a];
            pf.W[a] = (float)ps.W[a];
        }
        sh.partf[p] = pf;
    }
    for (int a = 0; a < 6; a++) fp[a] = 0.0;
}

}  // namespace lbp
