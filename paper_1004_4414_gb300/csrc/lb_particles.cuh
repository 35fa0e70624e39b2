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

// par: parity of this step.  The lists are rebuilt in this step when
// nl_flag[par] is set (by the MD of the previous step, or an init); the
// flag of the next step is cleared here, before this step's MD can set it.
static __global__ void k_step_begin(const BoxDev* __restrict__ boxes, int nb, Shared sh, int total_cells, int mslot_next,
                                    int par) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (sh.nl_flag[par])
        for (int i = tid; i < total_cells; i += gridDim.x * blockDim.x) sh.cell_count[i] = 0;
    if (tid == 0) {
        *sh.ev_count = 0;
        sh.nl_flag[par ^ 1] = 0;
    }
    if (tid < nb) {
        boxes[tid].mass_acc[mslot_next * 2 + 0] = 0.0;
        boxes[tid].mass_acc[mslot_next * 2 + 1] = 0.0;
    }
}

static __global__ void k_cell_count(const BoxDev* __restrict__ boxes, Shared sh, int NP, int par) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP || !sh.nl_flag[par]) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    atomicAdd(&sh.cell_count[cell_of(B, sh.part[p].X)], 1);
}

// one block per box: exclusive scan of the cell counts (offset by the box's
// first particle), cursors = starts
static __global__ void k_cell_scan(const BoxDev* __restrict__ boxes, Shared sh, int par) {
    if (!sh.nl_flag[par]) return;  // the whole block leaves together
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

static __global__ void k_cell_fill(const BoxDev* __restrict__ boxes, Shared sh, int NP, int par) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP || !sh.nl_flag[par]) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    const int pos = atomicAdd(&sh.cell_cursor[cell_of(B, sh.part[p].X)], 1);
    sh.cell_list[pos] = p;
}

// The particle a block (or warp) of a per-particle kernel takes: the i-th
// entry of the cell-sorted list, so that the blocks resident at one time
// work on neighbouring particles and share their cached fluid lines (a
// permutation of all particles from the first step on: the lists are built
// in every step after an init or import).
__device__ __forceinline__ int particle_at(const Shared& sh, int i) { return sh.cell_list[i]; }

// Neighbour list of p: every particle whose centre lies within nl_reach (a
// node owned before the move lies within R + |U| <= R + 1 of the new
// centre, lubrication acts below a gap of lub_cut, NL_SKIN of slack for the
// steps until the next build).  Built only in steps that rebuild the lists;
// the positions of the build are kept in xnl.
// One warp per particle; lane k scans cell k of the 3x3x3 block around p.
// FP32 distances against a slightly larger radius give a superset of the
// exact list, which is harmless for both users (claims and pair forces).
// The list is sorted by particle index, so the pair-force sums do not
// depend on the order in which the cells were filled.
constexpr int NLIST_WARPS = 4;
static __global__ void __launch_bounds__(32 * NLIST_WARPS) k_nlist(const BoxDev* __restrict__ boxes, Shared sh, int NP,
                                                                     int par) {
    __shared__ int s_ids[NLIST_WARPS][NL_MAX];
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * NLIST_WARPS + wib;
    if (p >= NP || !sh.nl_flag[par]) return;  // the whole warp leaves together
    const BoxDev& B = boxes[sh.pbox[p]];
    const PartStateF pf = sh.partf[p];
    if (lane < 3) sh.xnl[(size_t)p * 3 + lane] = pf.X[lane];
    const float reach = (float)nl_reach(B.rb, B.lub_cut);
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
// One block per particle p, its warps sharing the scan: record every node
// around X_p whose solid/fluid status or owner changes.  A node belongs to the particle whose
// centre is nearest among those within R (|x - X|^2 <= R^2, minimum image);
// ties go to the lower index.  Events: covered (fluid -> p), uncovered
// (p -> fluid), transfer (q -> p, no fluid involved).  Distances are FP32
// (relative to p, from the FP32 particle copy) unless they fall within
// `band` of R^2, where the FP64 value, evaluated without contraction as in a
// plain sequential evaluation, decides.  FP64 is slow on this GPU, so it is
// kept off the common path.
constexpr int DETECT_WARPS = 4, DETECT_QUEUE = 256;
// FP64 inside test of node (gx, gy, gz) for particle q: the squared centre
// distance if the node is inside, else -1.  Out of line so that the rare
// calls (FP32 undecided within a band of the surface, or a node near a second
// particle) branch to it instead of being predicated into every candidate's
// instruction stream: FP64 instructions issue at 1/16 of the FP32 rate here.
static __device__ __noinline__ double exact_inside(const BoxDev& B, const PartState* __restrict__ part, int q,
                                                   int gx, int gy, int gz) {
    const double* C = part[q].X;
    const double dx = mimg((double)gx - C[0], (double)B.nx), dy = mimg((double)gy - C[1], (double)B.ny),
                 dz = mimg((double)gz - C[2], (double)B.nz);
    return inside_shape(B, dx, dy, dz, part[q].E) ? dist2_nc(dx, dy, dz) : -1.0;
}

static __global__ void __launch_bounds__(32 * DETECT_WARPS, 6) k_remap_detect(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    __shared__ int s_queue[DETECT_WARPS][DETECT_QUEUE];  // annulus candidates of the fast path
    // the close list, built by each warp for itself
    __shared__ float s_rq[DETECT_WARPS][NL_MAX][3];  // X_q - X_p, minimum image
    __shared__ int s_nid[DETECT_WARPS][NL_MAX];
    __shared__ int s_cl[DETECT_WARPS][NL_MAX];  // entries of neighbours within 2R (+ slack)
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // in index order: the cell-sorted order measured 3 % slower here
    const int p = blockIdx.x;
    if (p >= NP) return;  // the whole block leaves together
    const int b = sh.pbox[p];
    const BoxDev& B = boxes[b];
    const PartStateF pf = sh.partf[p];
    // FP32 distances (spheres) or quadratic forms (spheroids) decide away
    // from the surface, the FP64 test (inside_shape) within a band of it
    const bool sph = B.aspect == 1.0;
    const float R = B.det_rb;
    const float Lf[3] = {(float)B.nx, (float)B.ny, (float)B.nz};
    const int nn = sh.nlist_n[p];
    // A node inside p can also be inside q only if |X_q - X_p| <= 2R (R the
    // bounding radius): those neighbours (the close list; 0.05 of slack
    // covers the FP32 centres) decide the claims of nodes inside p.  A node
    // p owned but left may lie within 2R + 1.5 of q, so that rare case scans
    // the whole list.
    const float rcl = 2.0f * R + 0.05f;
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
    const float reach = R + 1.5f;
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
    // window coordinates by multiplies when every coordinate of the window
    // lies within [-n, 2n) (always for a centre in the box and a reach below
    // the box edge; a centre that has run away, in an unstable state, takes
    // the division, whose wrap is valid for any coordinate)
    bool near = true;
    for (int a = 0; a < 3; a++) near = near && lo[a] >= -dims[a] && lo[a] <= 2 * dims[a] - span[a];
    const WinDiv wd(span[0], span[1], total < 65536 && near);
    // FP32 decisions away from the surface, the FP64 test within a band of
    // it (the box constants are set on the host; FP64 is slow on this GPU)
    const float Rf2o = B.det_reach2, R2f = B.det_R2, band = B.det_band;
    const float qlim = B.det_qlim;  // no node beyond this is inside q
    // spheroid prefilter: F = R^2 (d.e)^2 + c^2 (|d|^2 - (d.e)^2) against
    // R^2 c^2 in FP32; FP64 decides within sband
    float ex_ = 0.f, ey_ = 0.f, ez_ = 0.f;
    if (!sph) {
        const double* Ep = sh.part[p].E;
        ex_ = (float)Ep[0];
        ey_ = (float)Ep[1];
        ez_ = (float)Ep[2];
    }
    const float R2s = B.det_sR2, c2s = B.det_sc2, R2c2 = B.det_sR2c2, sband = B.det_sband;
    // one candidate node (kx, ky, kz) of the window: probe computes its
    // offsets from the centre and loads its owner (the only global load),
    // decide finds whether its status or owner changes (have), with its node
    // index, old and new owner; full scans probe several candidates before
    // deciding any, so that their loads are in flight together
    struct Cand {
        float fx, fy, fz, d2f;
        int n, own, gx, gy, gz;
        bool ok;
    };
    auto probe = [&](int kx, int ky, int kz) -> Cand {
        Cand c;
        c.fx = mimgf((float)kx - off[0], Lf[0]);
        c.fy = mimgf((float)ky - off[1], Lf[1]);
        c.fz = mimgf((float)kz - off[2], Lf[2]);
        c.d2f = c.fx * c.fx + c.fy * c.fy + c.fz * c.fz;
        c.ok = c.d2f <= Rf2o;
        c.gx = wd.wrap(lo[0] + kx, B.nx);
        c.gy = wd.wrap(lo[1] + ky, B.ny);
        c.gz = wd.wrap(lo[2] + kz, B.nz);
        c.n = c.gx + B.nx * (c.gy + B.ny * c.gz);
        c.own = c.ok ? __ldg(B.owner + c.n) : OWN_WALL;
        return c;
    };
    auto decide = [&](const Cand& c, bool& have, int& node, int& ev_old, int& ev_new) {
        if (!c.ok || c.own == OWN_WALL) return;
        const float fx = c.fx, fy = c.fy, fz = c.fz, d2f = c.d2f;
        const int gx = c.gx, gy = c.gy, gz = c.gz, own = c.own;
        // FP64 inside tests (exact_inside) where FP32 cannot decide; d2p is
        // the squared centre distance to p once known (the claim goes to the
        // nearest centre)
        double d2p = -1.0;
        bool inside;
        const float gap = sph ? d2f - R2f : [&] {
            const float sf = fx * ex_ + fy * ey_ + fz * ez_;
            return R2s * sf * sf + c2s * (d2f - sf * sf) - R2c2;
        }();
        if (fabsf(gap) > (sph ? band : sband)) {
            inside = gap < 0.0f;
        } else {
            d2p = exact_inside(B, sh.part, p, gx, gy, gz);
            inside = d2p >= 0.0;
        }
        if (!(inside || own == p)) return;
        bool other = false, anyone = false;
        const int nk = inside ? ncl : nn;
        for (int kk = 0; kk < nk; kk++) {
            const int k = inside ? s_cl[wib][kk] : kk;
            const float ex = mimgf(fx - s_rq[wib][k][0], Lf[0]);
            const float ey = mimgf(fy - s_rq[wib][k][1], Lf[1]);
            const float ez = mimgf(fz - s_rq[wib][k][2], Lf[2]);
            if (ex * ex + ey * ey + ez * ez > qlim) continue;
            const int q = s_nid[wib][k];
            const double d2q = exact_inside(B, sh.part, q, gx, gy, gz);
            if (d2q >= 0.0) {
                anyone = true;
                if (inside) {
                    if (d2p < 0.0) d2p = exact_inside(B, sh.part, p, gx, gy, gz);
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
        node = c.n;
    };
    // the events of 32 candidates, appended to the event list
    auto emit = [&](bool have, int node, int ev_old, int ev_new) {
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
    };
    // Fast path.  If the nodes p owns are exactly those inside p at the
    // position of the last remap X_ref (no other particle was within 2R
    // then: flag exact), and no other particle is within 2R now (ncl = 0),
    // then every node whose status changes through p lies in the annulus
    // R - delta < |x - X| <= R + delta, delta = |X - X_ref|: a node inside
    // p now but not before is farther than R - delta from X, a node inside
    // before but not now is within R + delta.  Only that annulus is scanned
    // (0.1 of slack covers the FP32 centre); the per-node decision is the
    // same as in the full scan, so the events are the same.  Spheres only.
    // delta from the FP32 copies: their error (~L 2^-24) is far inside the
    // 0.1 of slack
    float dref2 = 0.f;
    {
        const float* Xr = sh.xref + (size_t)p * 3;
        for (int a = 0; a < 3; a++) {
            const float v = mimgf(pf.X[a] - Xr[a], Lf[a]);
            dref2 += v * v;
        }
    }
    const float delta = sqrtf(dref2);
    bool fits = true;  // the window covers less than half of each axis (no wrap onto itself)
    for (int a = 0; a < 3; a++) fits = fits && 2 * span[a] < dims[a] && span[a] < 1024;
    const bool fast = sph && fits && ncl == 0 && sh.exact[p] && delta < 0.5f;
    if (!fits) {
        // a window that wraps onto itself (a box edge below twice the
        // window): every window node, two candidates per lane per round,
        // probed before either is decided
        constexpr int SU = 2;
        for (int base = wib * 32 * SU; base < total; base += 32 * SU * DETECT_WARPS) {
            Cand c[SU];
#pragma unroll
            for (int u = 0; u < SU; u++) {
                const int idx = base + u * 32 + lane;
                if (idx < total) {
                    int kx, ky, kz;
                    wd.split(idx, kx, ky, kz);
                    c[u] = probe(kx, ky, kz);
                } else {
                    c[u].ok = false;
                }
            }
#pragma unroll
            for (int u = 0; u < SU; u++) {
                int ev_old = 0, ev_new = 0, node = 0;
                bool have = false;
                decide(c[u], have, node, ev_old, ev_new);
                emit(have, node, ev_old, ev_new);
            }
        }
    } else {
        // rows (ky, kz) of the window, one per lane; the shell to scan (the
        // annulus of the fast path, else the ball of radius reach, with 0.01
        // of slack over the FP32 reach test) crosses a row in at most two x
        // intervals, whose nodes go to a per-warp queue
        const float r_out = fast ? R + delta + 0.1f : reach + 0.01f;
        const float r_in = fast ? fmaxf(R - delta - 0.1f, 0.0f) : 0.0f;
        int* q = s_queue[wib];
        const int nrows = span[1] * span[2];
        for (int rb = wib * 32; rb < nrows; rb += 32 * DETECT_WARPS) {
            const int row = rb + lane;
            int l0 = 0, h0 = -1, l1 = 0, h1 = -1;
            int ky = 0, kz = 0;
            if (row < nrows) {
                int kx_;
                wd.split(row * span[0], kx_, ky, kz);
                const float fy = (float)ky - off[1], fz = (float)kz - off[2];
                const float p2 = fy * fy + fz * fz;
                const float o2 = r_out * r_out - p2;
                if (o2 >= 0.0f) {
                    const float ao = sqrtf(o2);
                    const float i2 = r_in * r_in - p2;
                    // kx with |kx - off0| <= ao, minus |kx - off0| < ai
                    const int xl = max(0, (int)ceilf(off[0] - ao)), xh = min(span[0] - 1, (int)floorf(off[0] + ao));
                    if (i2 > 0.0f) {
                        const float ai = sqrtf(i2);
                        l0 = xl;
                        h0 = min(xh, (int)ceilf(off[0] - ai) - 1);
                        l1 = max(xl, (int)floorf(off[0] + ai) + 1);
                        h1 = xh;
                    } else {
                        l0 = xl;
                        h0 = xh;
                    }
                }
            }
            const int c0 = h0 >= l0 ? h0 - l0 + 1 : 0, c1 = h1 >= l1 ? h1 - l1 + 1 : 0;
            const int cnt = c0 + c1;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            // queue in chunks that fit: entries kx | ky << 10 | kz << 20
            for (int done = 0; done < tot; done += DETECT_QUEUE) {
                int pos = incl - cnt - done;
                for (int k = 0; k < cnt; k++, pos++) {
                    if (pos < 0 || pos >= DETECT_QUEUE) continue;
                    const int kx = k < c0 ? l0 + k : l1 + (k - c0);
                    q[pos] = kx | (ky << 10) | (kz << 20);
                }
                __syncwarp();
                const int nq = min(DETECT_QUEUE, tot - done);
                // two entries per lane per round, probed before either is decided
                for (int base = 0; base < nq; base += 64) {
                    Cand c[2];
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int j = base + u * 32 + lane;
                        if (j < nq) {
                            const int e = q[j];
                            c[u] = probe(e & 1023, (e >> 10) & 1023, e >> 20);
                        } else {
                            c[u].ok = false;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        int ev_old = 0, ev_new = 0, node = 0;
                        bool have = false;
                        decide(c[u], have, node, ev_old, ev_new);
                        emit(have, node, ev_old, ev_new);
                    }
                }
                __syncwarp();
            }
        }
    }
    // the reference position of the next remap, and whether p then owns
    // exactly the nodes inside it (no other particle within 2R); after every
    // warp has read the old values
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; a++) sh.xref[(size_t)p * 3 + a] = pf.X[a];
        sh.exact[p] = ncl == 0 ? 1 : 0;
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

// D3Q19 vectors as bit fields (2 bits per direction, value + 1), for a
// direction known only at run time (one per lane) without a memory lookup
__host__ __device__ constexpr uint64_t dir_bits(int a) {
    uint64_t v = 0;
    for (int i = 0; i < 19; i++) v |= (uint64_t)((a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i))) + 1) << (2 * i);
    return v;
}
__device__ __forceinline__ int dvec(int a, int i) {
    constexpr uint64_t B0 = dir_bits(0), B1 = dir_bits(1), B2 = dir_bits(2);
    const uint64_t b = a == 0 ? B0 : (a == 1 ? B1 : B2);
    return (int)((b >> (2 * i)) & 3u) - 1;
}
__device__ __forceinline__ void node_xyz(const BoxDev& B, int n, int& x, int& y, int& z) {
    x = n % B.nx;
    const int r = n / B.nx;
    y = r % B.ny;
    z = r / B.ny;
}
// node at (x + dx, y + dy, z + dz), |d| <= 1 per axis, periodic
__device__ __forceinline__ int node_off(const BoxDev& B, int x, int y, int z, int dx, int dy, int dz) {
    return wrap1(x + dx, B.nx) + B.nx * (wrap1(y + dy, B.ny) + B.ny * wrap1(z + dz, B.nz));
}

// Cover / uncover.  PAR is the parity of the coming fused step.  Before an
// even step f_i of a node sits in its own slot i; before an odd step it sits
// in slot opp(i) of the neighbour x - c_i, whatever that neighbour's status
// (the even step stores a population reflected at a solid node in that
// node's slot).  So a status change moves nothing: a covered node gives the
// momentum of its populations to the particle, an uncovered node gets
// f^eq(rho_new, u_s) in the same places, and the particle loses the
// momentum of the created fluid.  One warp per event, lane i takes
// direction i (1..18).
template <class P, int PAR>
static __global__ void k_remap_apply(const BoxDev* __restrict__ boxes, Shared sh, int rc, int mslot_cur) {
    using R = typename P::real;
    using R2 = typename Real2<R>::type;
    using S2 = typename P::st2;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int cnt = ev_total(sh);
    const int i = lane;
    const bool act = i >= 1 && i <= 18;
    const int ix = act ? dvec(0, i) : 0, iy = act ? dvec(1, i) : 0, iz = act ? dvec(2, i) : 0;
    const int io = act ? opp(i) : 0;
    for (int e = warp; e < cnt; e += nwarps) {
        const int4 ev = sh.events[e];
        const int w = ev.x, old = ev.z, nw = ev.w;
        if (old != OWN_FLUID && nw != OWN_FLUID) continue;  // transfer between particles (warp-uniform)
        const BoxDev& B = boxes[ev.y];
        const Pop<P> pop(B);
        int x, y, z;
        node_xyz(B, w, x, y, z);
        // the pair of f_i of w before the coming step
        S2* const at = act ? (PAR == 0 ? pop.pair(i, w) : pop.pair(io, node_off(B, x, y, z, -ix, -iy, -iz))) : nullptr;
        if (old == OWN_FLUID) {
            // covered: the particle gains the momentum of the node's fluid
            double m0 = 0.0, m1 = 0.0, m2 = 0.0;
            if (act) {
                R a, b;
                pop.ld2(at, i, a, b);
                const double v = (double)a + (double)b;
                m0 = v * ix;
                m1 = v * iy;
                m2 = v * iz;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                m0 += __shfl_xor_sync(FULL, m0, o);
                m1 += __shfl_xor_sync(FULL, m1, o);
                m2 += __shfl_xor_sync(FULL, m2, o);
            }
            if (lane == 0) {
                atomicAdd(&sh.counters[ev.y * 2 + 0], 1ull);
                double r[3];
                node_rel(B, sh, w, nw, r);
                const double mom[3] = {m0, m1, m2};
                add_force_torque(sh, nw, r, mom);
            }
        } else {
            // uncovered (Eqs. eqn_rho_neu and masscorr): the mean density of
            // the neighbours that were fluid, times the mass-correction
            // factor; f = f^eq(rho_new, u_s) of the particle that left it
            const R2* __restrict__ rcur2 = rpair<R>(B.rho[rc]);
            R s0 = R(0), s1 = R(0);
            int c = 0;
            if (act) {
                const int m = node_off(B, x, y, z, ix, iy, iz);
                if (!old_solid(B, m)) {
                    const R2 v = rcur2[m];
                    s0 = v.x;
                    s1 = v.y;
                    c = 1;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(FULL, s0, o);
                s1 += __shfl_xor_sync(FULL, s1, o);
                c += __shfl_xor_sync(FULL, c, o);
            }
            double corr[2] = {1.0, 1.0};
            if (B.c0 != 0.0) {
                const double rsum = B.rho_init[0] + B.rho_init[1];
                for (int k = 0; k < 2; k++)
                    corr[k] = 1.0 - B.c0 * (rsum / B.rho_init[k]) * (B.mass_acc[mslot_cur * 2 + k] - B.mass0[k]) /
                                        (double)B.N;
            }
            const R rb0 = c ? s0 / (R)c : (R)B.rho_init[0], rb1 = c ? s1 / (R)c : (R)B.rho_init[1];
            const R rn0 = (R)((double)rb0 * corr[0]), rn1 = (R)((double)rb1 * corr[1]);
            const PartState ps = sh.part[old];
            const double r[3] = {mimg((double)x - ps.X[0], B.nx), mimg((double)y - ps.X[1], B.ny),
                                 mimg((double)z - ps.X[2], B.nz)};
            const R us[3] = {(R)(ps.U[0] + ps.W[1] * r[2] - ps.W[2] * r[1]),
                             (R)(ps.U[1] + ps.W[2] * r[0] - ps.W[0] * r[2]),
                             (R)(ps.U[2] + ps.W[0] * r[1] - ps.W[1] * r[0])};
            // the 18 moving populations; the density rho_new (set by
            // k_remap_finish) makes the rest population rho_new minus them
            if (act) {
                R q0, q1;
                pop.st2(at, i, feq_rt<R>(i, rn0, us[0], us[1], us[2]), feq_rt<R>(i, rn1, us[0], us[1], us[2]), q0, q1);
            }
            if (lane == 0) {
                sh.ev_rho[(size_t)e * 2 + 0] = (double)rn0;
                sh.ev_rho[(size_t)e * 2 + 1] = (double)rn1;
                atomicAdd(&sh.counters[ev.y * 2 + 1], 1ull);
                // the particle loses the momentum of the created fluid
                // (Eq. eqn_ladd_vernichtenunderzeugen, sign from conservation)
                const double rs = (double)rn0 + (double)rn1;
                const double F[3] = {-rs * (double)us[0], -rs * (double)us[1], -rs * (double)us[2]};
                add_force_torque(sh, old, r, F);
            }
        }
    }
}

// shell flag of node (x, y, z): solid with a fluid D3Q19 neighbour
__device__ __forceinline__ void shell_update_at(const BoxDev& B, int x, int y, int z) {
    const int n = x + B.nx * (y + B.ny * z);
    const uint8_t f = B.flags[n];
    if (!(f & FL_SOLID)) return;
    bool shl = false;
#pragma unroll
    for (int i = 1; i < 19; i++)
        if (!(B.flags[node_off(B, x, y, z, cx(i), cy(i), cz(i))] & FL_SOLID)) shl = true;
    B.flags[n] = FL_SOLID | (shl ? FL_SHELL : 0);
}
__device__ __forceinline__ void shell_update(const BoxDev& B, int n) {
    int x, y, z;
    node_xyz(B, n, x, y, z);
    shell_update_at(B, x, y, z);
}

// After the events: densities of the event nodes, shell flags around them,
// and the particles whose shell lists must be rebuilt.  One warp per event:
// lane 0 takes the event node, lane i (1..18) its neighbour w + c_i.
template <class R>
static __global__ void k_remap_finish(const BoxDev* __restrict__ boxes, Shared sh, int rc) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const int cnt = ev_total(sh);
    const int i = lane;
    const int ix = i <= 18 ? dvec(0, i) : 0, iy = i <= 18 ? dvec(1, i) : 0, iz = i <= 18 ? dvec(2, i) : 0;
    for (int e = warp; e < cnt; e += nwarps) {
        const int4 ev = sh.events[e];
        const BoxDev& B = boxes[ev.y];
        const int w = ev.x;
        R* rcur = reinterpret_cast<R*>(B.rho[rc]);
        int x, y, z;
        node_xyz(B, w, x, y, z);
        if (lane == 0) {
            if (ev.z == OWN_FLUID) {
                rcur[2 * (size_t)w] = R(0);
                rcur[2 * (size_t)w + 1] = R(0);
            } else if (ev.w == OWN_FLUID) {
                rcur[2 * (size_t)w] = (R)sh.ev_rho[(size_t)e * 2 + 0];
                rcur[2 * (size_t)w + 1] = (R)sh.ev_rho[(size_t)e * 2 + 1];
            }
            B.evmark[w] = 0;
            // the particles whose shell lists this event can change: the old
            // and new owner of w and the owners of its solid neighbours
            // (their fluid-neighbour masks)
            if (ev.z >= 0) sh.shell_dirty[ev.z] = 1;
            if (ev.w >= 0) sh.shell_dirty[ev.w] = 1;
        }
        if (i <= 18) {
            const int nx_ = wrap1(x + ix, B.nx), ny_ = wrap1(y + iy, B.ny), nz_ = wrap1(z + iz, B.nz);
            const int n = nx_ + B.nx * (ny_ + B.ny * nz_);
            if (i >= 1) {
                const int o = B.owner[n];
                if (o >= 0) sh.shell_dirty[o] = 1;
            }
            // A solid node left without fluid neighbours takes density 0: the
            // fused step may have counted reflected populations in it while it
            // was a shell node, and no later pass rewrites it (the particle's
            // Shan-Chen force reads it through its shell neighbours).
            shell_update_at(B, nx_, ny_, nz_);
            if (B.flags[n] == FL_SOLID) {
                rcur[2 * (size_t)n] = R(0);
                rcur[2 * (size_t)n + 1] = R(0);
            }
        }
    }
}

// ------------------------------------------------------- virtual fluid
// Shell nodes get the mean density of their fluid neighbours plus the
// particle colour on red (Delta rho > 0) or blue (Delta rho < 0) (Sec. IV).
// One block per particle; its warps share the work.  The per-particle shell
// list (node, mask of fluid neighbours, x | y << 16, z) is kept across steps
// and rebuilt only when an event touched the particle (shell_dirty).
constexpr int SHELL_WARPS = 4;
constexpr int SHELL_CUBE = 8192;  // flag bytes of a rebuild window with its one-node ring
constexpr int SHELL_QW = 256;     // shell-flagged candidates a warp can queue in a rebuild
constexpr int SHELL_KQ = 4;       // queued candidates per thread whose owner loads are in flight together
template <class R>
static __global__ void __launch_bounds__(32 * SHELL_WARPS) k_shell_density(const BoxDev* __restrict__ boxes, Shared sh,
                                                                          int rc, int NP) {
    using R2 = typename Real2<R>::type;
    __shared__ int s_cnt[SHELL_WARPS];
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((int)blockIdx.x >= NP) return;  // the whole block leaves together
    const int p = particle_at(sh, blockIdx.x);
    const BoxDev& B = boxes[sh.pbox[p]];
    const PartStateF pf = sh.partf[p];
    R2* __restrict__ r2 = rpair<R>(B.rho[rc]);
    const uint8_t* __restrict__ flags = B.flags;
    const int32_t* __restrict__ owner = B.owner;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int nxy = nx * ny;
    const float R_ = (float)B.rb;  // bounding radius (the radius for spheres)
    const R col = (R)sh.color[p];
    const int scap = sh.shell_cap;
    int4* __restrict__ slist = sh.shell_list + (size_t)p * scap;
    auto finish = [&](int n, R s0, R s1, int cnt) {
        R r0 = s0 / (R)cnt, r1 = s1 / (R)cnt;
        if (col > R(0)) r0 += col;
        else if (col < R(0)) r1 -= col;
        r2[n] = mk2<R2>(r0, r1);
    };
    if (!sh.shell_dirty[p]) {
        // No event near p since its list was built: the shell nodes and
        // their fluid-neighbour masks are unchanged, only the densities are
        // new (the whole block takes this branch together).  Two entries
        // per thread per round: all their density loads are issued before
        // either node is written.
        const int ns = sh.shell_n[p];
        constexpr int NT = 32 * SHELL_WARPS;
        for (int k0 = threadIdx.x; k0 < ns; k0 += 2 * NT) {
            R s0[2] = {R(0), R(0)}, s1[2] = {R(0), R(0)};
            int nk[2] = {0, 0};
            unsigned fm[2] = {0u, 0u};
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int k = k0 + NT * u;
                if (k >= ns) continue;
                const int4 e = slist[k];
                const int n = e.x;
                const unsigned fmask = (unsigned)e.y;
                nk[u] = n;
                fm[u] = fmask;
                const int gx = e.z & 0xffff, gy = (int)((unsigned)e.z >> 16), gz = e.w;
                const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
                const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
                const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    if (!((fmask >> i) & 1u)) continue;
                    const int m = n + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) +
                                  (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) + (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
                    const R2 v = r2[m];
                    s0[u] += v.x;
                    s1[u] += v.y;
                }
            }
#pragma unroll
            for (int u = 0; u < 2; u++)
                if (k0 + NT * u < ns) finish(nk[u], s0[u], s1[u], __popc(fm[u]));
        }
        return;
    }
    // Rebuild: every shell node of p lies within R of its centre, so the
    // window of nodes within R + 0.5 (the slack covers the FP32 centre) is
    // scanned; the shell flag and the owner decide.  No FP64 here: it is
    // slow on this GPU.
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
    const float lim = reach * reach;
    constexpr int NT = 32 * SHELL_WARPS;
    // Rebuild from a shared-memory copy of the window's flags (windows of
    // up to SHELL_CUBE nodes with their ring, which covers R + 0.5 <= 8 or
    // so): the candidates are tested in shared memory, and only the shell-
    // flagged ones within reach go to a queue, in window order.  Their
    // owners are loaded together, a block-wide prefix gives each shell node
    // of p its list position (window order again, so the list does not
    // depend on timing), and the fluid-neighbour masks come from the copy.
    // Three dependent rounds of global loads (flags, owners, densities)
    // instead of one per candidate.  Larger windows, or a queue that would
    // overflow, take the two-pass scan below.
    const int wx = span[0] + 2, wy = span[1] + 2, wz = span[2] + 2;
    // window (with its ring) coordinates by multiplies when they all lie
    // within [-n, 2n) (a centre that has run away takes the division)
    bool near = true;
    for (int a = 0; a < 3; a++) near = near && lo[a] - 1 >= -dims[a] && lo[a] + 1 <= 2 * dims[a] - span[a];
    const bool nodiv = total < 65536 && near;
    const WinDiv wd(span[0], span[1], nodiv);
    if (wx * wy * wz <= SHELL_CUBE) {
        const WinDiv wc(wx, wy, nodiv);
        __shared__ uint8_t s_fl[SHELL_CUBE];
        __shared__ int s_q[SHELL_WARPS][SHELL_QW];
        __shared__ int s_qn[SHELL_WARPS];
        __shared__ int s_kc[SHELL_KQ][SHELL_WARPS];
        const int cube = wx * wy * wz;
        for (int i = threadIdx.x; i < cube; i += NT) {
            int a, b, c;
            wc.split(i, a, b, c);
            const int gx = wc.wrap(lo[0] - 1 + a, nx), gy = wc.wrap(lo[1] - 1 + b, ny), gz = wc.wrap(lo[2] - 1 + c, nz);
            s_fl[i] = __ldg(flags + gx + nx * (gy + ny * gz));
        }
        __syncthreads();
        // warp w queues the candidates of the contiguous range [beg, end)
        const int per = (total + SHELL_WARPS - 1) / SHELL_WARPS;
        const int beg = wib * per, end = min(total, beg + per);
        int qn = 0;
        for (int b0 = beg; b0 < end; b0 += 32) {
            const int idx = b0 + lane;
            bool c = false;
            if (idx < end) {
                int kx, ky, kz;
                wd.split(idx, kx, ky, kz);
                const float dx = mimgf((float)kx - off[0], (float)nx), dy = mimgf((float)ky - off[1], (float)ny),
                            dz = mimgf((float)kz - off[2], (float)nz);
                c = dx * dx + dy * dy + dz * dz <= lim && (s_fl[(kx + 1) + wx * ((ky + 1) + wy * (kz + 1))] & FL_SHELL);
            }
            const unsigned m = __ballot_sync(FULL, c);
            const int at = qn + __popc(m & ((1u << lane) - 1u));
            if (c && at < SHELL_QW) s_q[wib][at] = idx;
            qn += __popc(m);
        }
        if (lane == 0) s_qn[wib] = qn;
        __syncthreads();
        int qoff[SHELL_WARPS + 1];
        bool fits = true;
        qoff[0] = 0;
#pragma unroll
        for (int w = 0; w < SHELL_WARPS; w++) {
            fits = fits && s_qn[w] <= SHELL_QW;
            qoff[w + 1] = qoff[w] + s_qn[w];
        }
        if (fits) {  // the same for the whole block
            const int nq = qoff[SHELL_WARPS];
            int listed = 0;  // shell nodes of p listed so far
            for (int q0 = 0; q0 < nq; q0 += SHELL_KQ * NT) {
                int kidx[SHELL_KQ];
                bool tk[SHELL_KQ];
#pragma unroll
                for (int k = 0; k < SHELL_KQ; k++) {
                    const int q = q0 + k * NT + threadIdx.x;
                    kidx[k] = -1;
                    tk[k] = false;
                    if (q < nq) {
                        int w = 0;
#pragma unroll
                        for (int v = 1; v < SHELL_WARPS; v++) w += q >= qoff[v];
                        const int idx = s_q[w][q - qoff[w]];
                        int kx, ky, kz;
                        wd.split(idx, kx, ky, kz);
                        const int gx = wd.wrap(lo[0] + kx, nx), gy = wd.wrap(lo[1] + ky, ny), gz = wd.wrap(lo[2] + kz, nz);
                        kidx[k] = idx;
                        tk[k] = __ldg(owner + gx + nx * (gy + ny * gz)) == p;
                    }
                }
                unsigned bm[SHELL_KQ];
#pragma unroll
                for (int k = 0; k < SHELL_KQ; k++) {
                    bm[k] = __ballot_sync(FULL, tk[k]);
                    if (lane == 0) s_kc[k][wib] = __popc(bm[k]);
                }
                __syncthreads();
                int before = listed, round = 0;
#pragma unroll
                for (int k = 0; k < SHELL_KQ; k++)
#pragma unroll
                    for (int w = 0; w < SHELL_WARPS; w++) round += s_kc[k][w];
#pragma unroll
                for (int k = 0; k < SHELL_KQ; k++) {
                    int pos = before;
#pragma unroll
                    for (int w = 0; w < SHELL_WARPS; w++)
                        if (w < wib) pos += s_kc[k][w];
                    pos += __popc(bm[k] & ((1u << lane) - 1u));
                    if (tk[k]) {
                        // virtual density and list entry of the shell node
                        const int idx = kidx[k];
                        int kx, ky, kz;
                        wd.split(idx, kx, ky, kz);
                        const int gx = wd.wrap(lo[0] + kx, nx), gy = wd.wrap(lo[1] + ky, ny), gz = wd.wrap(lo[2] + kz, nz);
                        const int n = gx + nx * (gy + ny * gz);
                        const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
                        const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
                        const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
                        const uint8_t* const fc = s_fl + (kx + 1) + wx * ((ky + 1) + wy * (kz + 1));
                        R s0 = R(0), s1 = R(0);
                        unsigned fmask = 0;
#pragma unroll
                        for (int i = 1; i < 19; i++) {
                            if (fc[cx(i) + wx * (cy(i) + wy * cz(i))] & FL_SOLID) continue;
                            const int m = n + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) +
                                          (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) + (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
                            const R2 v = r2[m];
                            s0 += v.x;
                            s1 += v.y;
                            fmask |= 1u << i;
                        }
                        if (pos < scap) slist[pos] = make_int4(n, (int)fmask, (int)((unsigned)gx | ((unsigned)gy << 16)), gz);
                        finish(n, s0, s1, __popc(fmask));
                    }
#pragma unroll
                    for (int w = 0; w < SHELL_WARPS; w++) before += s_kc[k][w];
                }
                listed += round;
                __syncthreads();  // s_kc is rewritten by the next round
            }
            if (threadIdx.x == 0) {
                sh.shell_n[p] = listed < scap ? listed : scap;
                if (listed > scap) set_err(sh.err, ERR_OVERFLOW);
                else sh.shell_dirty[p] = 0;
            }
            return;
        }
    }
    // candidate idx of the window: a shell node of p?
    auto test = [&](int idx, int& n, int& cxy, int& cz) -> bool {
        if (idx >= total) return false;
        const int kx = idx % span[0], ky = (idx / span[0]) % span[1], kz = idx / (span[0] * span[1]);
        const float dx = mimgf((float)kx - off[0], (float)nx), dy = mimgf((float)ky - off[1], (float)ny),
                    dz = mimgf((float)kz - off[2], (float)nz);
        if (!(dx * dx + dy * dy + dz * dz <= lim)) return false;
        const int gx = wrapi(lo[0] + kx, nx), gy = wrapi(lo[1] + ky, ny), gz = wrapi(lo[2] + kz, nz);
        n = gx + nx * (gy + ny * gz);
        cxy = (int)((unsigned)gx | ((unsigned)gy << 16));
        cz = gz;
        return (__ldg(flags + n) & FL_SHELL) && __ldg(owner + n) == p;
    };
    // virtual density of one shell node n of p, and its entry k of p's
    // shell list (node, mask of fluid neighbours, coordinates)
    auto process = [&](int n, int cxy, int gz, int k) {
        const int gx = cxy & 0xffff, gy = (int)((unsigned)cxy >> 16);
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
                const R2 v = r2[m];
                s0 += v.x;
                s1 += v.y;
                cnt++;
                fmask |= 1u << i;
            }
        }
        if (k < scap) slist[k] = make_int4(n, (int)fmask, cxy, gz);
        finish(n, s0, s1, cnt);
    };
    // Two passes over the same candidates, each warp taking chunks of 32 SU
    // in turn: the first counts each warp's shell nodes, the second lists
    // them after those of the lower warps, so the list order does not
    // depend on timing.  The second pass finds the flags and owners in L1.
    constexpr int SU = 4, CH = 32 * SU;
    int mine = 0;
    for (int base = wib * CH; base < total; base += CH * SHELL_WARPS) {
        bool tk[SU];
        int nu[SU], cu[SU], zu[SU];
#pragma unroll
        for (int u = 0; u < SU; u++) tk[u] = test(base + u * 32 + lane, nu[u], cu[u], zu[u]);
#pragma unroll
        for (int u = 0; u < SU; u++) mine += __popc(__ballot_sync(FULL, tk[u]));
    }
    if (lane == 0) s_cnt[wib] = mine;
    __syncthreads();
    int pos = 0, done = 0;
#pragma unroll
    for (int w = 0; w < SHELL_WARPS; w++) {
        if (w < wib) pos += s_cnt[w];
        done += s_cnt[w];
    }
    for (int base = wib * CH; base < total; base += CH * SHELL_WARPS) {
        bool tk[SU];
        int nu[SU], cu[SU], zu[SU];
#pragma unroll
        for (int u = 0; u < SU; u++) tk[u] = test(base + u * 32 + lane, nu[u], cu[u], zu[u]);
#pragma unroll
        for (int u = 0; u < SU; u++) {
            const unsigned m = __ballot_sync(FULL, tk[u]);
            if (tk[u]) process(nu[u], cu[u], zu[u], pos + __popc(m & ((1u << lane) - 1u)));
            pos += __popc(m);
        }
    }
    if (threadIdx.x == 0) {
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
// IMPL: the box may use the implicit velocity update; its links then also
// sum the drag tensor Z = sum_links sum_c 6 zeta_j rho^c(x) a a^T with
// a = (c_j, r x c_j) (upper triangle into zdrag).
constexpr int COUPLE_THREADS = 128;
constexpr int NZ = 21;  // entries of the symmetric 6 x 6 drag tensor
// five resident blocks per SM without the implicit update's drag tensor (96
// registers, 16 B of spills): 2 % faster than the compiler's 124 registers;
// three with it (154 registers)
template <class P, bool IMPL>
static __global__ void __launch_bounds__(COUPLE_THREADS, IMPL ? 3 : 5)
    k_couple(const BoxDev* __restrict__ boxes, Shared sh, int rc, int rn, int mslot, int par, int reflect) {
    using R = typename P::real;
    using S2 = typename P::st2;
    using R2 = typename Real2<R>::type;
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NRED = 8 + (IMPL ? NZ : 0);
    __shared__ R s_red[COUPLE_THREADS / 32][NRED];
    const int p = particle_at(sh, blockIdx.x);
    const BoxDev& B = boxes[sh.pbox[p]];
    const Pop<P> pop(B);
    const auto& ps = part_ptr<R>(sh)[p];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int nxy = nx * ny;
    const R2* __restrict__ rcur2 = rpair<R>(B.rho[rc]);
    R2* __restrict__ rnext2 = rpair<R>(B.rho[rn]);
    double* __restrict__ mass_acc = B.mass_acc;
    const R rho0 = (R)B.rho0, irho0 = R(1) / (R)B.rho0, g = (R)B.g;
    const R wax = (R)B.scw_axis, wdg = (R)B.scw_diag;
    const R Lx = (R)nx, Ly = (R)ny, Lz = (R)nz;
    const R X0 = (R)ps.X[0], X1 = (R)ps.X[1], X2 = (R)ps.X[2];
    const R U0 = (R)ps.U[0], U1 = (R)ps.U[1], U2 = (R)ps.U[2];
    const R W0 = (R)ps.W[0], W1 = (R)ps.W[1], W2 = (R)ps.W[2];
    // the reflected pair f*_j (j = opp(i)) of the link from m = s + c_i to
    // s belongs after an even step in slot j of s, after an odd step in
    // slot i of m; unreflected it sits in the other of the two
    const bool at_s = (par == 0) == (reflect != 0);
    R acc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R dm0 = R(0), dm1 = R(0);
    R zz[IMPL ? NZ : 1];
#pragma unroll
    for (int e = 0; e < (IMPL ? NZ : 1); e++) zz[e] = R(0);
    const bool impl = IMPL && B.implicit;
    // the shell nodes found by k_shell_density in this step, one per thread
    const int ns = sh.shell_n[p];
    const int4* __restrict__ list = sh.shell_list + (size_t)p * sh.shell_cap;
    for (int k = threadIdx.x; k < ns; k += COUPLE_THREADS) {
        const int4 e = list[k];
        const int s = e.x;
        const unsigned fmask = (unsigned)e.y;  // bit i: s + c_i is fluid (a link)
        const int gx = e.z & 0xffff, gy = (int)((unsigned)e.z >> 16), gz = e.w;
        const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
        const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
        const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
        auto nb = [&](int i) -> int {
            return s + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) + (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) +
                   (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
        };
        // s relative to the centre
        const R rs0 = mimg_r<R>((R)gx - X0, Lx), rs1 = mimg_r<R>((R)gy - X1, Ly), rs2 = mimg_r<R>((R)gz - X2, Lz);
        const R2 rss = __ldg(rcur2 + s);
        R sr0 = R(0), sr1 = R(0), sr2 = R(0), sb0 = R(0), sb1 = R(0), sb2 = R(0);
        // directions in three groups of six: the loads of a group (the
        // densities of the neighbours, the populations of the links) are
        // issued before any of its stores
#pragma unroll
        for (int grp = 0; grp < 3; grp++) {
            R2 rm[6];
            S2 raw[6];
#pragma unroll
            for (int t = 0; t < 6; t++) {
                const int i = 1 + 6 * grp + t;
                const int m = nb(i);
                rm[t] = __ldg(rcur2 + m);
                if ((fmask >> i) & 1u) raw[t] = *(at_s ? pop.pair(opp(i), s) : pop.pair(i, m));
            }
#pragma unroll
            for (int t = 0; t < 6; t++) {
                const int i = 1 + 6 * grp + t;
                // Shan-Chen: Psi of every neighbour (fluid, virtual or interior)
                const R w = is_axis(i) ? wax : wdg;
                const R pr = w * psi_of<R>(rm[t].x, rho0, irho0);
                const R pb = w * psi_of<R>(rm[t].y, rho0, irho0);
                sr0 += pr * (R)cx(i);
                sr1 += pr * (R)cy(i);
                sr2 += pr * (R)cz(i);
                sb0 += pb * (R)cx(i);
                sb1 += pb * (R)cy(i);
                sb2 += pb * (R)cz(i);
                if (!((fmask >> i) & 1u)) continue;
                // link from the fluid node m to s; c_j = -c_i; midpoint s + c_i / 2
                const int m = nb(i);
                const R r0 = rs0 + R(0.5) * (R)cx(i), r1 = rs1 + R(0.5) * (R)cy(i), r2 = rs2 + R(0.5) * (R)cz(i);
                const R us0 = U0 + W1 * r2 - W2 * r1, us1 = U1 + W2 * r0 - W0 * r2, us2 = U2 + W0 * r1 - W1 * r0;
                const R cu6 =
                    -R(6) * wgt<R>(i) * (us0 * (R)cx(i) + us1 * (R)cy(i) + us2 * (R)cz(i));
                R fs[2], wall[2], dr[2] = {R(0), R(0)};
                if constexpr (P::dev) {
                    fs[0] = pop.dev_to_f(0, i, raw[t].x);
                    fs[1] = pop.dev_to_f(1, i, raw[t].y);
                } else {
                    fs[0] = raw[t].x;
                    fs[1] = raw[t].y;
                }
                wall[0] = cu6 * rm[t].x;
                wall[1] = cu6 * rm[t].y;
                if (cu6 != R(0) || !reflect) {
                    S2 q = raw[t];
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
                    // reflect = 0 moves the value to the other slot
                    S2* const to = (at_s == (reflect != 0)) ? pop.pair(opp(i), s) : pop.pair(i, m);
                    *to = q;
                    red_add2<R>(rnext2 + m, reflect ? dr[0] : dr[0] + fs[0], reflect ? dr[1] : dr[1] + fs[1]);
                    dm0 += dr[0];
                    dm1 += dr[1];
                }
                const R mag = (R(2) * fs[0] - wall[0]) + (R(2) * fs[1] - wall[1]);
                const R F0 = -mag * (R)cx(i), F1 = -mag * (R)cy(i), F2 = -mag * (R)cz(i);
                acc[0] += F0;
                acc[1] += F1;
                acc[2] += F2;
                acc[3] += r1 * F2 - r2 * F1;
                acc[4] += r2 * F0 - r0 * F2;
                acc[5] += r0 * F1 - r1 * F0;
                if constexpr (IMPL) {
                    if (impl) {
                        // a = (c_j, r x c_j), c_j = -c_i
                        const R a[6] = {-(R)cx(i), -(R)cy(i), -(R)cz(i), -(r1 * (R)cz(i) - r2 * (R)cy(i)),
                                        -(r2 * (R)cx(i) - r0 * (R)cz(i)), -(r0 * (R)cy(i) - r1 * (R)cx(i))};
                        const R kz = R(6) * wgt<R>(i) * (rm[t].x + rm[t].y);
                        int e = 0;
#pragma unroll
                        for (int u = 0; u < 6; u++)
#pragma unroll
                            for (int v = u; v < 6; v++) zz[e++] += kz * a[u] * a[v];
                    }
                }
            }
        }
        // the Shan-Chen force of the virtual fluid at s on the particle
        // (Eq. eqn_shan_chen_particle), torque (s - X) x F
        const R psr = psi_of<R>(rss.x, rho0, irho0), psb = psi_of<R>(rss.y, rho0, irho0);
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
        if constexpr (IMPL) {
#pragma unroll
            for (int e = 0; e < NZ; e++) zz[e] += __shfl_xor_sync(FULL, zz[e], o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 6; a++) s_red[wib][a] = acc[a];
        s_red[wib][6] = dm0;
        s_red[wib][7] = dm1;
        if constexpr (IMPL) {
#pragma unroll
            for (int e = 0; e < NZ; e++) s_red[wib][8 + e] = zz[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        const int a = threadIdx.x;
        R v = s_red[0][a];
#pragma unroll
        for (int w = 1; w < COUPLE_THREADS / 32; w++) v += s_red[w][a];
        // the only writer of this particle's accumulators in this kernel
        if (a < 6) sh.force[(size_t)p * 6 + a] += (double)v;
        else if (a < 8) {
            if (v != R(0)) atomicAdd(&mass_acc[mslot * 2 + (a - 6)], (double)v);
        } else if (impl) {
            sh.zdrag[(size_t)p * NZ + (a - 8)] = (double)v;
        }
    }
}

// Implicit update, fluid side (after k_md_solve): every link of particle p
// gets the wall term of the velocity change, -6 zeta_j rho^c(x) a.dV, on
// the reflected pair that the next step reads, and the same change enters
// rho(t+1) of the fluid node and the step's fluid mass.  The links, the
// positions and the densities are those k_couple used in this step, so the
// fluid's momentum change is the opposite of -Z dV on the particle.
template <class P>
static __global__ void __launch_bounds__(COUPLE_THREADS)
    k_couple_correct(const BoxDev* __restrict__ boxes, Shared sh, int rc, int rn, int mslot, int par, int reflect) {
    using R = typename P::real;
    using S2 = typename P::st2;
    using R2 = typename Real2<R>::type;
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ R s_red[COUPLE_THREADS / 32][2];
    const int p = particle_at(sh, blockIdx.x);
    const BoxDev& B = boxes[sh.pbox[p]];
    if (!B.implicit || B.fixed) return;  // the whole block leaves together
    const Pop<P> pop(B);
    const auto& ps = part_ptr<R>(sh)[p];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int nxy = nx * ny;
    const R2* __restrict__ rcur2 = rpair<R>(B.rho[rc]);
    R2* __restrict__ rnext2 = rpair<R>(B.rho[rn]);
    const R Lx = (R)nx, Ly = (R)ny, Lz = (R)nz;
    const R X0 = (R)ps.X[0], X1 = (R)ps.X[1], X2 = (R)ps.X[2];
    R dV[6];
#pragma unroll
    for (int u = 0; u < 6; u++) dV[u] = (R)sh.dv[(size_t)p * 6 + u];
    const bool at_s = (par == 0) == (reflect != 0);
    R dm0 = R(0), dm1 = R(0);
    const int ns = sh.shell_n[p];
    const int4* __restrict__ list = sh.shell_list + (size_t)p * sh.shell_cap;
    for (int k = threadIdx.x; k < ns; k += COUPLE_THREADS) {
        const int4 e = list[k];
        const int s = e.x;
        const unsigned fmask = (unsigned)e.y;
        const int gx = e.z & 0xffff, gy = (int)((unsigned)e.z >> 16), gz = e.w;
        const int oxm = gx == 0 ? nx - 1 : -1, oxp = gx == nx - 1 ? -(nx - 1) : 1;
        const int oym = gy == 0 ? (ny - 1) * nx : -nx, oyp = gy == ny - 1 ? -(ny - 1) * nx : nx;
        const int ozm = gz == 0 ? (nz - 1) * nxy : -nxy, ozp = gz == nz - 1 ? -(nz - 1) * nxy : nxy;
        const R rs0 = mimg_r<R>((R)gx - X0, Lx), rs1 = mimg_r<R>((R)gy - X1, Ly), rs2 = mimg_r<R>((R)gz - X2, Lz);
#pragma unroll
        for (int i = 1; i < 19; i++) {
            if (!((fmask >> i) & 1u)) continue;
            const int m = s + (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) + (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) +
                          (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
            const R r0 = rs0 + R(0.5) * (R)cx(i), r1 = rs1 + R(0.5) * (R)cy(i), r2 = rs2 + R(0.5) * (R)cz(i);
            // a.dV with a = (c_j, r x c_j), c_j = -c_i
            const R ad = -((R)cx(i) * dV[0] + (R)cy(i) * dV[1] + (R)cz(i) * dV[2]) -
                         ((r1 * (R)cz(i) - r2 * (R)cy(i)) * dV[3] + (r2 * (R)cx(i) - r0 * (R)cz(i)) * dV[4] +
                          (r0 * (R)cy(i) - r1 * (R)cx(i)) * dV[5]);
            const R2 rm = __ldg(rcur2 + m);
            const R d0 = R(6) * wgt<R>(i) * rm.x * ad, d1 = R(6) * wgt<R>(i) * rm.y * ad;
            // the slot k_couple wrote the reflected pair to
            S2* const to = (at_s == (reflect != 0)) ? pop.pair(opp(i), s) : pop.pair(i, m);
            S2 q = *to;
            if constexpr (P::dev) {
                q.x = pop.f_to_dev(0, i, pop.dev_to_f(0, i, q.x) - d0);
                q.y = pop.f_to_dev(1, i, pop.dev_to_f(1, i, q.y) - d1);
            } else {
                q.x -= d0;
                q.y -= d1;
            }
            *to = q;
            red_add2<R>(rnext2 + m, -d0, -d1);
            dm0 -= d0;
            dm1 -= d1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm0 += __shfl_xor_sync(FULL, dm0, o);
        dm1 += __shfl_xor_sync(FULL, dm1, o);
    }
    if (lane == 0) {
        s_red[wib][0] = dm0;
        s_red[wib][1] = dm1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        R v = s_red[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < COUPLE_THREADS / 32; w++) v += s_red[w][threadIdx.x];
        if (v != R(0)) atomicAdd(&B.mass_acc[mslot * 2 + threadIdx.x], (double)v);
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

// Pair forces (Hertz contact and lubrication) on p into fpair; the velocity
// update adds them to the fluid's force.  One warp per particle, lane k
// takes the k-th entry of the (sorted) neighbour list; a fixed butterfly
// sums the lanes, so the result does not depend on timing.  Reads only the
// positions, velocities and neighbour lists, so it runs beside the fluid
// kernels of the step.
constexpr int MD_WARPS = 4;
static __global__ void __launch_bounds__(32 * MD_WARPS) k_md_pair(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const unsigned FULL = 0xffffffffu;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((int)(blockIdx.x * MD_WARPS + wib) >= NP) return;  // the whole warp leaves together
    const int p = particle_at(sh, blockIdx.x * MD_WARPS + wib);
    const BoxDev& B = boxes[sh.pbox[p]];
    double F[3] = {0.0, 0.0, 0.0};
    const int nn = sh.nlist_n[p];
    if (lane < nn) {
        // FP32 prefilter: only pairs within contact or lubrication range
        // (centre distance below 2 R_b + lub_cut, with slack for the FP32
        // positions) take the FP64 force
        const int q = sh.nlist[(size_t)p * NL_MAX + lane];
        const PartStateF a = sh.partf[p], b = sh.partf[q];
        const float dx = mimgf(a.X[0] - b.X[0], (float)B.nx), dy = mimgf(a.X[1] - b.X[1], (float)B.ny),
                    dz = mimgf(a.X[2] - b.X[2], (float)B.nz);
        const float lim = 2.0f * (float)B.rb + (float)B.lub_cut + 0.01f;
        if (dx * dx + dy * dy + dz * dz < lim * lim) pair_force(B, sh.part[p], sh.part[q], F);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; a++) F[a] += __shfl_xor_sync(FULL, F[a], off);
    if (lane < 3) sh.fpair[(size_t)p * 3 + lane] = F[lane];
}

// The force and torque on p of this step: the fluid's part (k_couple and
// the remap events) is kept in force_last, then the pair forces are added.
__device__ __forceinline__ void total_force(const Shared& sh, int p, double f[6]) {
    const double* fp = &sh.force[(size_t)p * 6];
    for (int a = 0; a < 6; a++) {
        f[a] = fp[a];
        sh.force_last[(size_t)p * 6 + a] = f[a];
    }
    for (int a = 0; a < 3; a++) f[a] += sh.fpair[(size_t)p * 3 + a];
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

// the lists of the next step (parity par ^ 1) are rebuilt when p has moved
// more than NL_SKIN / 2 since the last build
__device__ __forceinline__ void nl_check(const BoxDev& B, const Shared& sh, int p, const PartStateF& pf, int par) {
    const float* xb = sh.xnl + (size_t)p * 3;
    const float dx = mimgf(pf.X[0] - xb[0], (float)B.nx), dy = mimgf(pf.X[1] - xb[1], (float)B.ny),
                dz = mimgf(pf.X[2] - xb[2], (float)B.nz);
    if (!(dx * dx + dy * dy + dz * dz <= 0.25f * NL_SKIN * NL_SKIN)) sh.nl_flag[par ^ 1] = 1;
}

// Solve A x = b for a 6 x 6 system by Gaussian elimination with partial
// pivoting; A (row-major) and b are overwritten.
__device__ __forceinline__ void solve6(double A[36], double b[6], double x[6]) {
    for (int col = 0; col < 6; col++) {
        int piv = col;
        for (int r = col + 1; r < 6; r++)
            if (fabs(A[6 * r + col]) > fabs(A[6 * piv + col])) piv = r;
        if (piv != col) {
            for (int v = 0; v < 6; v++) {
                const double t = A[6 * col + v];
                A[6 * col + v] = A[6 * piv + v];
                A[6 * piv + v] = t;
            }
            const double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < 6; r++) {
            const double f = A[6 * r + col] / A[6 * col + col];
            for (int v = col; v < 6; v++) A[6 * r + v] -= f * A[6 * col + v];
            b[r] -= f * b[col];
        }
    }
    for (int r = 5; r >= 0; r--) {
        double t = b[r];
        for (int v = r + 1; v < 6; v++) t -= A[6 * r + v] * x[v];
        x[r] = t / A[6 * r + r];
    }
}

// Velocity half of the MD step for handles where some box uses the implicit
// update (k_md_move then moves the particles, after k_couple_correct has
// given the fluid its share).  Implicit boxes: (M + Z) dV = (F, T) with
// M = diag(m, m, m, J, J, J) and the links' drag tensor Z of k_couple, then
// U += dU, omega += d omega (dV kept for k_couple_correct).  Other boxes: the
// explicit update of k_md_integrate.  Accumulators zeroed.
static __global__ void k_md_solve(const BoxDev* __restrict__ boxes, Shared sh, int NP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    double* fp = &sh.force[(size_t)p * 6];
    double ft[6];
    total_force(sh, p, ft);
    PartState ps = sh.part[p];
    double dv[6] = {0, 0, 0, 0, 0, 0};
    if (!B.fixed) {
        if (B.implicit) {
            double A[36], b[6];
            int e = 0;
            for (int u = 0; u < 6; u++)
                for (int v = u; v < 6; v++) {
                    const double z = sh.zdrag[(size_t)p * NZ + e++];
                    A[6 * u + v] = z;
                    A[6 * v + u] = z;
                }
            for (int u = 0; u < 3; u++) {
                A[7 * u] += B.mass;
                A[7 * (u + 3)] += B.inertia;
                b[u] = ft[u];
                b[u + 3] = ft[3 + u];
            }
            solve6(A, b, dv);
            for (int a = 0; a < 3; a++) {
                ps.U[a] += dv[a];
                ps.W[a] += dv[3 + a];
            }
        } else {
            if (B.aspect != 1.0) rotate_spheroid(B, ps.W, ps.E, ft + 3);
            for (int a = 0; a < 3; a++) {
                ps.U[a] += ft[a] / B.mass;
                if (B.aspect == 1.0) ps.W[a] += ft[3 + a] / B.inertia;
            }
        }
        if (!(ps.U[0] * ps.U[0] + ps.U[1] * ps.U[1] + ps.U[2] * ps.U[2] < 1.0)) set_err(sh.err, ERR_FAST_PARTICLE);
        sh.part[p] = ps;
    }
    for (int a = 0; a < 6; a++) {
        sh.dv[(size_t)p * 6 + a] = dv[a];
        fp[a] = 0.0;
    }
}

// Position half: X += U (periodic) and the FP32 copy.  par: parity of this step.
static __global__ void k_md_move(const BoxDev* __restrict__ boxes, Shared sh, int NP, int par) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    if (B.fixed) return;
    PartState ps = sh.part[p];
    const double L[3] = {(double)B.nx, (double)B.ny, (double)B.nz};
    PartStateF pf;
    for (int a = 0; a < 3; a++) {
        double xn = ps.X[a] + ps.U[a];
        xn -= L[a] * floor(xn / L[a]);
        if (xn >= L[a]) xn -= L[a];
        sh.part[p].X[a] = xn;
        pf.X[a] = (float)xn;
        pf.U[a] = (float)ps.U[a];
        pf.W[a] = (float)ps.W[a];
    }
    sh.partf[p] = pf;
    nl_check(B, sh, p, pf, par);
}

// leap-frog: U += F/m, omega += T/J (spheroids: rotate_spheroid), X += U
// (periodic); accumulators zeroed.  par: parity of this step.
static __global__ void k_md_integrate(const BoxDev* __restrict__ boxes, Shared sh, int NP, int par) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const BoxDev& B = boxes[sh.pbox[p]];
    double* fp = &sh.force[(size_t)p * 6];
    double ft[6];
    total_force(sh, p, ft);
    PartState ps = sh.part[p];
    if (!B.fixed) {
        const double L[3] = {(double)B.nx, (double)B.ny, (double)B.nz};
        if (B.aspect != 1.0) rotate_spheroid(B, ps.W, ps.E, ft + 3);
        for (int a = 0; a < 3; a++) {
            ps.U[a] += ft[a] / B.mass;
            if (B.aspect == 1.0) ps.W[a] += ft[3 + a] / B.inertia;
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
        nl_check(B, sh, p, pf, par);
    }
    for (int a = 0; a < 6; a++) fp[a] = 0.0;
}

}  // namespace lbp
