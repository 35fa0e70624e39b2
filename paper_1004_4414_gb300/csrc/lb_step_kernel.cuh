// lb_step_kernel.cuh -- the fused per-step kernel of the fluid: streaming
// with bounce-back, Shan-Chen force, cubic-equilibrium BGK collision, and the
// density field of the next step.
//
// Method (paper): Eq. eq:boltz with the BGK operator and the equilibrium of
// Eq. Equil at the velocity shifted by tau F / rho (Sec. II); the force of
// Eq. eqn_shan-chen-F with Psi of Eq. eqn_ref_dens over the 18 D3Q19 links;
// bounce-back at solid nodes (Eq. eqn_bounce-back).  The moving-wall term,
// the momentum exchange and the shell force on the particles are added
// afterwards by k_couple (lb_particles.cuh), which only touches the links
// at particle surfaces.
//
// GB300 design:
//   * Populations stay in place with the AA pattern.  Even steps: a node
//     reads its own 18 slots and writes f*_j to slot opp(j) of itself.  Odd
//     steps: it reads f_i from slot opp(i) of x - c_i and writes f*_j to slot
//     j of x + c_j.  A population whose stream target y = x + c_j is solid
//     belongs, reflected, in the slot the next step reads it from: slot j
//     of y after an even step (the odd step at x reads its f_opp(j) there),
//     slot opp(j) of x after an odd step.  So the loads of both parities
//     never depend on the status of a neighbour.  Each slot is read once and
//     written once per step; neighbour offsets are wrap-aware and computed
//     once per thread.
//   * The two components of a direction and node form one pair in memory
//     (8 bytes in FP32, 4 in 16-bit storage), so one load or store moves
//     both: a warp moves 32 consecutive pairs of one direction per access.
//     Every operation that is the same for both components is one packed
//     FP32 instruction on the pair (FADD2 / FMUL2 / FFMA2).  16-bit storage
//     stages the next plane's pairs in shared memory with cp.async while the
//     current plane is computed (StepStage below).
//   * Only the 18 moving populations are stored.  A node's rho^c is the
//     density field of the current step (the window fetches it for Psi
//     anyway), and its rest population f_0 = rho^c - sum_{i>=1} f_i stays at
//     the node: it enters only the density scatter.  So a fluid node moves
//     2 x 18 populations per step, and the density field is the state's
//     mass.
//   * Reflection (template flag BB).  BB = true: the kernel reads the solid
//     status of the 18 neighbours and selects each store's slot itself.
//     BB = false: it stores every population as if its target were fluid
//     (even steps slot opp(j) of x, odd steps slot j of y) and scatters it
//     to y's density; k_couple then moves each of these values to its
//     reflected slot, adds the moving-wall term and counts the value in x's
//     density.  This needs a link list that covers every fluid-solid link,
//     which the particles' shell lists do; boxes with static walls use
//     BB = true.  The moved-from slots are never read: the slot of x (even
//     steps) is read next by y, which is solid, and the slot of y (odd
//     steps) is refilled before y can become fluid again.
//   * A CTA owns a column tile of 32 x TY nodes (one warp per x row: all
//     population traffic is coalesced along x) and marches through a chunk
//     of z planes.  Psi and the node flags of the tile plus a one-node ring
//     sit in a three-plane shared-memory ring buffer.
//   * The force needs Psi of every neighbour at the same time level, so the
//     kernel produces rho(t+1) itself from the values it stores.  The values
//     a node sends are summed by destination group (dy, dz); the x shift is
//     a warp shuffle, the y shift a shared-memory exchange between rows and
//     the z shift free (each thread marches along its own column and keeps
//     the partial sums of three planes in registers).  Nodes whose whole
//     stencil lies in the tile are written with plain stores; tile-edge and
//     ring nodes are added with global reductions into a density buffer that
//     was zeroed at exactly those nodes during the previous step (ring of
//     three density buffers: current, next, to-zero).
#pragma once
#include <type_traits>

#include "lb_common.cuh"

namespace lbp {

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Psi = rho0 (1 - exp(-rho / rho0)); irho0 = 1 / rho0
template <class R>
__device__ __forceinline__ R psi_of(R rho, R rho0, R irho0) {
    if constexpr (sizeof(R) == 8) return rho0 * (1.0 - exp(-rho * irho0));
    else return rho0 * (1.0f - expf(-rho * irho0));
}

template <class R>
__device__ __forceinline__ const typename PartOf<R>::type* part_ptr(const Shared& sh) {
    if constexpr (sizeof(R) == 8) return sh.part;
    else return sh.partf;
}

template <class R>
__device__ __forceinline__ R mimg_r(R d, R L) {
    return d > R(0.5) * L ? d - L : (d < -R(0.5) * L ? d + L : d);
}

template <class R>
__device__ __forceinline__ void red_add(R* p, R v) {
    atomicAdd(p, v);
}
// both components of a density-ring pair (one vector reduction in FP32)
template <class R>
__device__ __forceinline__ void red_add2(typename Real2<R>::type* p, R a, R b) {
    if constexpr (sizeof(R) == 4) {
        atomicAdd(p, make_float2(a, b));
    } else {
        atomicAdd(&p->x, a);
        atomicAdd(&p->y, b);
    }
}

// Destination groups of the density scatter: (dy, dz) of a direction.
//   g: 0 (0,0) 1 (+1,0) 2 (-1,0) 3 (0,+1) 4 (0,-1) 5 (+1,+1) 6 (-1,-1)
//      7 (+1,-1) 8 (-1,+1)
__host__ __device__ constexpr int grp_of(int i) {
    constexpr int g[19] = {0, 0, 0, 1, 2, 3, 4, 1, 2, 2, 1, 3, 4, 4, 3, 5, 6, 7, 8};
    return g[i];
}
__host__ __device__ constexpr int grp_dy(int g) {
    constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return v[g];
}
__host__ __device__ constexpr int grp_dz(int g) {
    constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return v[g];
}
// groups with dy != 0 go through the shared-memory row exchange: index 0..5
__host__ __device__ constexpr int yb_of(int g) {
    constexpr int v[9] = {-1, 0, 1, -1, -1, 2, 3, 4, 5};
    return v[g];
}

// lattice vectors for a direction known only at run time (rare paths)
static __constant__ signed char kC[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                             {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                             {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                             {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

template <class R, int TY>
struct StepSmem {
    static constexpr int W2 = 34, H2 = TY + 2, PLANE = W2 * H2;
    static constexpr size_t psi_elems = (size_t)3 * 2 * PLANE;
    static constexpr size_t yb_elems = (size_t)6 * 2 * TY * 32;
    static constexpr size_t bytes = (psi_elems + yb_elems) * sizeof(R) + (size_t)3 * PLANE + 64;
};

// Staging of the next plane's populations (16-bit storage): each thread
// copies the 18 pairs its node reads in plane z + 1 into its own column of
// a [18][32 TY] shared array with cp.async while plane z is computed, so
// that the population loads of the step overlap the work of the plane
// before (the 16-byte-aligned array follows the window).  Measured at
// 256^3: 3 % faster for FP16 storage, 2 % slower for FP32, which keeps
// its loads in registers.
template <class P, int TY>
struct StepStage {
    static constexpr bool on = P::dev;
    static constexpr size_t offset = (StepSmem<typename P::real, TY>::bytes + 15) & ~(size_t)15;
    static constexpr size_t bytes = on ? (size_t)18 * 32 * TY * sizeof(typename P::st2) : 0;
    static constexpr size_t smem = offset + bytes;
};
__device__ __forceinline__ void cp_async_sz(void* sdst, const void* gsrc, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// T1: every box has tau^r = tau^b = 1, where BGK gives f* = f^eq: the
// loaded populations then only feed the moments and need not stay live.
// Resident CTAs per SM for the FP32 / 16-bit tau = 1 kernel: five of 128
// threads at TY = 4 (96 registers, 20 warps), three of 256 at TY = 8 (80
// registers, 24 warps); measured at 256^3, five small CTAs beat three and
// six (and four or more at TY = 8, which spills).  Otherwise two.
template <class P, bool T1>
constexpr int step_min_blocks(int ty) {
    return ty > 8 ? 1 : (!(T1 && sizeof(typename P::real) == 4) ? 2 : (ty == 4 ? 5 : 3));
}
template <class P, int PAR, int TY, bool T1, bool BB>
static __global__ void __launch_bounds__(32 * TY, step_min_blocks<P, T1>(TY))
    k_step(const BoxDev* __restrict__ boxes, const TileDev* __restrict__ tiles, Shared sh, int rc, int rn, int rz,
           int mslot) {
    using R = typename P::real;
    using S = typename P::st;
    using SM = StepSmem<R, TY>;
    constexpr int W2 = SM::W2, H2 = SM::H2;
    using R2 = typename Real2<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Psi window: (Psi^r, Psi^b) pairs, [3 slots][H2][W2]
    R2* s_psi2 = reinterpret_cast<R2*>(smem_raw);
    R* s_yb = reinterpret_cast<R*>(smem_raw) + SM::psi_elems;          // [6][2][TY][32]
    uint8_t* s_flg = reinterpret_cast<uint8_t*>(s_yb + SM::yb_elems);  // [3 slots][H2][W2]
    __shared__ double s_red[2][TY];

    const TileDev T = tiles[blockIdx.x];
    const BoxDev& B = boxes[T.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = B.N;
    const int nxy = nx * ny;
    using S2 = typename P::st2;
    const R2* __restrict__ rcur = rpair<R>(B.rho[rc]);
    R* __restrict__ rnext = reinterpret_cast<R*>(B.rho[rn]);  // component c of node m: rnext[2 m + c]
    R2* __restrict__ rnext2 = rpair<R>(B.rho[rn]);
    R2* __restrict__ rzero = rpair<R>(B.rho[rz]);
    const uint8_t* __restrict__ gflags = B.flags;
    const Pop<P> pop(B);
    const R rho0 = (R)B.rho0, irho0 = R(1) / (R)B.rho0, g = (R)B.g;
    const R tau0 = (R)B.tau[0], tau1 = (R)B.tau[1], itau0 = (R)B.inv_tau[0], itau1 = (R)B.inv_tau[1];
    const R wax = (R)B.scw_axis, wdg = (R)B.scw_diag;
    const R bfx = (R)B.body[0], bfy = (R)B.body[1], bfz = (R)B.body[2];
    const int velmode = B.vel_mode;

    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
    const int w = T.w, h = T.h, d = T.d, x0 = T.x0, y0 = T.y0, z0 = T.z0;
    const bool active = lx < w && ly < h;
    const int x = active ? x0 + lx : x0, y = active ? y0 + ly : y0;
    // wrap-aware neighbour offsets along x and y
    const int oxm = (x == 0) ? nx - 1 : -1, oxp = (x == nx - 1) ? -(nx - 1) : 1;
    const int oym = (y == 0) ? (ny - 1) * nx : -nx, oyp = (y == ny - 1) ? -(ny - 1) * nx : nx;
    const int nxyc = x + nx * y;  // in-plane index

    auto PSI2 = [&](int s, int r, int k) -> R2& { return s_psi2[(s * H2 + r) * W2 + k]; };
    auto FLG = [&](int s, int r, int k) -> uint8_t& { return s_flg[(s * H2 + r) * W2 + k]; };
    // this thread's node in a window plane; neighbours at constant offsets
    const int tofs = (ly + 1) * W2 + lx + 1;
    R2* const s_yb2 = reinterpret_cast<R2*>(s_yb);  // row exchange: [6][TY][32] pairs
    auto YB2 = [&](int q, int r, int k) -> R2& { return s_yb2[(q * TY + r) * 32 + k]; };

    // The window of a plane: Psi and flags of the tile (one node per
    // thread) and of its one-node ring (thread tid < nring takes ring node
    // (ring_r, ring_k)); ring positions do not depend on the plane.
    const int nring = 2 * (w + 2) + 2 * h;
    int ring_r = 0, ring_k = 0, ring_xy = 0;
    if (tid < nring) {
        if (tid < w + 2) {
            ring_r = 0;
            ring_k = tid;
        } else if (tid < 2 * (w + 2)) {
            ring_r = h + 1;
            ring_k = tid - (w + 2);
        } else if (tid < 2 * (w + 2) + h) {
            ring_k = 0;
            ring_r = tid - 2 * (w + 2) + 1;
        } else {
            ring_k = w + 1;
            ring_r = tid - 2 * (w + 2) - h + 1;
        }
        int gx = x0 + ring_k - 1, gy = y0 + ring_r - 1;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        ring_xy = gx + nx * gy;
    }
    // raw window values of one plane, fetched ahead of their use
    struct WinRaw {
        R a0, a1, b0, b1;
        uint8_t af, bf;
    };
    auto fetch_window = [&](int zz) {
        WinRaw v{R(0), R(0), R(0), R(0), 0, 0};
        const int gz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        const int pb = nxy * gz;
        if (active) {
            const int n = pb + nxyc;
            const R2 r = rcur[n];
            v.a0 = r.x;
            v.a1 = r.y;
            v.af = gflags[n];
        }
        if (tid < nring) {
            const int n = pb + ring_xy;
            const R2 r = rcur[n];
            v.b0 = r.x;
            v.b1 = r.y;
            v.bf = gflags[n];
        }
        return v;
    };
    auto store_window = [&](const WinRaw& v, int s) {
        if (active) {
            PSI2(s, ly + 1, lx + 1) = mk2<R2>(psi_of<R>(v.a0, rho0, irho0), psi_of<R>(v.a1, rho0, irho0));
            FLG(s, ly + 1, lx + 1) = v.af;
        }
        if (tid < nring) {
            PSI2(s, ring_r, ring_k) = mk2<R2>(psi_of<R>(v.b0, rho0, irho0), psi_of<R>(v.b1, rho0, irho0));
            FLG(s, ring_r, ring_k) = v.bf;
        }
    };
    auto load_window = [&](int zz, int s) { store_window(fetch_window(zz), s); };

    // rolling slots of planes z-1, z, z+1
    int sm_ = 0, sc_ = 1, sp_ = 2;
    load_window(z0 - 1, sm_);
    // the densities of the own node in planes z and z + 1: the window
    // fetches them anyway, and they are the node's rho^r and rho^b
    R rq0[2], rq1[2];
    {
        const WinRaw v0 = fetch_window(z0);
        store_window(v0, sc_);
        rq0[0] = v0.a0;
        rq0[1] = v0.a1;
        const WinRaw v1 = fetch_window(z0 + 1);
        store_window(v1, sp_);
        rq1[0] = v1.a0;
        rq1[1] = v1.a1;
    }
    R2 acc[3];  // own-column partial densities of planes z-1, z, z+1
#pragma unroll
    for (int k = 0; k < 3; k++) acc[k] = p2(R(0));
    R2 msum = p2(R(0));  // fluid mass sent (own precision: Eq. masscorr uses small differences)
    __syncthreads();

    // this thread's 18 staged pairs: s_stage[(i - 1) * 32 TY + tid]
    using ST = StepStage<P, TY>;
    S2* const s_stage = reinterpret_cast<S2*>(smem_raw + ST::offset);
    // issue the copies of the pairs node (x, y, zz) reads (if it is fluid)
    auto stage = [&](int zz, bool fl) {
        if constexpr (ST::on) {
            if (fl) {
                const int zm = (zz == 0) ? (nz - 1) * nxy : -nxy, zp = (zz == nz - 1) ? -(nz - 1) * nxy : nxy;
                const int nn = nxyc + nxy * zz;
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    const int j = opp(i);
                    const int o = (cx(j) < 0 ? oxm : (cx(j) > 0 ? oxp : 0)) + (cy(j) < 0 ? oym : (cy(j) > 0 ? oyp : 0)) +
                                  (cz(j) < 0 ? zm : (cz(j) > 0 ? zp : 0));
                    const S2* p = PAR == 0 ? pop.pair(i, nn) : pop.pair(j, nn + o);
                    cp_async_sz(s_stage + (i - 1) * (32 * TY) + tid, p, (int)sizeof(S2));
                }
            }
            cp_async_commit();
        }
    };
    stage(z0, active && !(FLG(sc_, ly + 1, lx + 1) & FL_SOLID));

    for (int z = z0; z < z0 + d; z++) {
        // window of plane z + 2, fetched now and stored at the end of this
        // plane, so that its load latency hides behind the plane's work
        const bool more = z + 1 < z0 + d;
        WinRaw ahead{R(0), R(0), R(0), R(0), 0, 0};
        if (more) ahead = fetch_window(z + 2);
        const int ozm = (z == 0) ? (nz - 1) * nxy : -nxy, ozp = (z == nz - 1) ? -(nz - 1) * nxy : nxy;
        const int n = nxyc + nxy * z;
        // offset of the neighbour x + c_i (i known at compile time)
        auto off = [&](int i) -> int {
            return (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) + (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) +
                   (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
        };
        // offset of the node (x, y + dy, z + dz) of scatter group q
        auto yz = [&](int q) -> int {
            const int dy = grp_dy(q), dz = grp_dz(q);
            return (dy < 0 ? oym : (dy > 0 ? oyp : 0)) + (dz < 0 ? ozm : (dz > 0 ? ozp : 0));
        };

        // window planes z - 1, z, z + 1 at this thread's node
        const R2* const wp[3] = {s_psi2 + sm_ * SM::PLANE + tofs, s_psi2 + sc_ * SM::PLANE + tofs,
                                 s_psi2 + sp_ * SM::PLANE + tofs};
        const uint8_t* const wf[3] = {s_flg + sm_ * SM::PLANE + tofs, s_flg + sc_ * SM::PLANE + tofs,
                                      s_flg + sp_ * SM::PLANE + tofs};
        const uint8_t fl = active ? wf[1][0] : FL_SOLID;
        const bool fluid = active && !(fl & FL_SOLID);
        unsigned smask = 0;  // bit i: x + c_i is solid
        // component pairs (red, blue) throughout: one packed instruction
        // per operation for both components
        R2 f[19];
        R2 rho = p2(R(1)), ux = p2(R(0)), uy = p2(R(0)), uz = p2(R(0));
        if (fluid) {
            // ------------------------------------------------- fluid node
            if constexpr (BB) {
#pragma unroll
                for (int i = 1; i < 19; i++)
                    smask |= (unsigned)(wf[cz(i) + 1][cy(i) * W2 + cx(i)] & FL_SOLID) << i;
            }
            if constexpr (ST::on) {
                // staged during the previous plane (this thread's own copies)
                cp_async_wait_all();
#pragma unroll
                for (int i = 1; i < 19; i++) pop.cvt2(s_stage[(i - 1) * (32 * TY) + tid], i, f[i].x, f[i].y);
            } else {
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    // even steps: own slot i; odd steps: slot opp(i) of x - c_i
                    const S2* p = PAR == 0 ? pop.pair(i, n) : pop.pair(opp(i), n + off(opp(i)));
                    pop.ld2(p, i, f[i].x, f[i].y);
                }
            }
            // rho^c is the density field (the sum of the values the previous
            // step sent here); the rest population is rho^c minus the 18
            // moving ones and is needed only for tau != 1
            R2 rs = p2(R(0)), jx = p2(R(0)), jy = p2(R(0)), jz = p2(R(0));
#pragma unroll
            for (int i = 1; i < 19; i++) {
                if constexpr (!T1) rs = padd(rs, f[i]);
                if (cx(i) > 0) jx = padd(jx, f[i]);
                if (cx(i) < 0) jx = psub(jx, f[i]);
                if (cy(i) > 0) jy = padd(jy, f[i]);
                if (cy(i) < 0) jy = psub(jy, f[i]);
                if (cz(i) > 0) jz = padd(jz, f[i]);
                if (cz(i) < 0) jz = psub(jz, f[i]);
            }
            rho = mk2<R2>(rq0[0], rq0[1]);
            f[0] = T1 ? p2(R(0)) : psub(rho, rs);
            // Shan-Chen force F^c = -g Psi^c(x) sum_i W_i Psi^cbar(x + c_i) c_i:
            // one pair load per neighbour, swapped so that each component
            // meets the other one's Psi
            R2 Fx, Fy, Fz;
            {
                R2 sx = p2(R(0)), sy = p2(R(0)), sz = p2(R(0));
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    const R2 pp = wp[cz(i) + 1][cy(i) * W2 + cx(i)];
                    const R2 q = mk2<R2>(pp.y, pp.x);
                    const R w = is_axis(i) ? wax : wdg;
                    if (cx(i)) sx = pfma(q, p2(cx(i) > 0 ? w : -w), sx);
                    if (cy(i)) sy = pfma(q, p2(cy(i) > 0 ? w : -w), sy);
                    if (cz(i)) sz = pfma(q, p2(cz(i) > 0 ? w : -w), sz);
                }
                const R2 pc = pmul(p2(-g), wp[1][0]);
                Fx = pfma(pc, sx, pmul(rho, p2(bfx)));
                Fy = pfma(pc, sy, pmul(rho, p2(bfy)));
                Fz = pfma(pc, sz, pmul(rho, p2(bfz)));
            }
            const R2 it2 = mk2<R2>(itau0, itau1);
            const R2 rt = pmul(rho, it2);
            const R iden = R(1) / (rt.x + rt.y);
            const R2 qx = pmul(jx, it2), qy = pmul(jy, it2), qz = pmul(jz, it2);
            const R2 ir = mk2<R2>(R(1) / rho.x, R(1) / rho.y);
            const R2 bx_ = velmode ? pmul(jx, ir) : p2((qx.x + qx.y) * iden);
            const R2 by_ = velmode ? pmul(jy, ir) : p2((qy.x + qy.y) * iden);
            const R2 bz_ = velmode ? pmul(jz, ir) : p2((qz.x + qz.y) * iden);
            const R2 tir = pmul(mk2<R2>(tau0, tau1), ir);
            ux = pfma(Fx, tir, bx_);
            uy = pfma(Fy, tir, by_);
            uz = pfma(Fz, tir, bz_);
            const R rtot = rho.x + rho.y;
            const R vx = jx.x + jx.y, vy = jy.x + jy.y, vz = jz.x + jz.y;
            if (!(rho.x > R(0)) || !(rho.y > R(0)) || !(vx * vx + vy * vy + vz * vz < R(0.25) * rtot * rtot))
                set_err(sh.err, ERR_UNSTABLE);
        }
        // the moments have consumed every staged pair of this node: stage
        // plane z + 1 (its flags are in the window) behind this plane's work
        if (more) stage(z + 1, active && !(wf[2][0] & FL_SOLID));

        const unsigned FULL = 0xffffffffu;
        // per-group partial sums of the pairs this node sends (mid: no x
        // move; up / dn: to x + 1 / x - 1); after the x shuffle mid[g] holds
        // everything that arrives in this column
        R2 mid[9], up[5], dn[5];
#pragma unroll
        for (int q = 0; q < 9; q++) mid[q] = p2(R(0));
#pragma unroll
        for (int q = 0; q < 5; q++) up[q] = dn[q] = p2(R(0));
        if (fluid) {
            const R2 itc = T1 ? p2(R(1)) : mk2<R2>(itau0, itau1);
            const R2 omt = T1 ? p2(R(0)) : psub(p2(R(1)), itc);
            const R2 uu = pfma(ux, ux, pfma(uy, uy, pmul(uz, uz)));
            const R2 a0 = pfma(p2(R(-1.5)), uu, p2(R(1)));
            const R2 rw1 = pmul(rho, p2(wgt<R>(1))), rw7 = pmul(rho, p2(wgt<R>(7)));
            R2 resid = p2(R(0)), fe_sum = p2(R(0)), self = p2(R(0));
            // store the pair f*_j where the next step reads it.  Stream target
            // y = x + c_j fluid: even steps slot opp(j) of x, odd steps slot j
            // of y.  Target solid (bounce-back, f_opp(j) of x at t+1): even
            // steps slot j of y, which the odd step at x reads for direction
            // opp(j); odd steps slot opp(j) of x.
            auto send = [&](auto JC, R2 fs) {
                constexpr int j = decltype(JC)::value;
                const bool solid = BB && ((smask >> j) & 1u);
                S2* p;
                if (PAR == 0) p = solid ? pop.pair(j, n + off(j)) : pop.pair(opp(j), n);
                else p = solid ? pop.pair(opp(j), n) : pop.pair(j, n + off(j));
                R2 q;
                pop.st2(p, j, fs.x, fs.y, q.x, q.y);
                if constexpr (P::dev) resid = padd(resid, psub(fs, q));
                const R2 qf = solid ? p2(R(0)) : q;
                if constexpr (BB) self = padd(self, solid ? q : p2(R(0)));
                constexpr int gq = grp_of(j);
                if (cx(j) == 0) mid[gq] = padd(mid[gq], qf);
                else if (cx(j) > 0) up[gq] = padd(up[gq], qf);
                else dn[gq] = padd(dn[gq], qf);
            };
            // equilibria of opposite pairs share their even part:
            // f^eq_(+/-) = zeta rho (E +/- O), E = 1 - 3/2 u^2 + 9/2 cu^2,
            // O = cu (3 + 9/2 (cu^2 - u^2))
            auto pair = [&](auto JC, R2 cu) {
                constexpr int j = decltype(JC)::value;
                const R2 rw = is_axis(j) ? rw1 : rw7;
                const R2 cu2 = pmul(cu, cu);
                const R2 E = pfma(p2(R(4.5)), cu2, a0);
                const R2 O = pmul(cu, pfma(p2(R(4.5)), psub(cu2, uu), p2(R(3))));
                const R2 fep = pmul(rw, padd(E, O)), fem = pmul(rw, psub(E, O));
                fe_sum = padd(fe_sum, padd(fep, fem));
                if constexpr (T1) {
                    send(std::integral_constant<int, j>{}, fep);
                    send(std::integral_constant<int, opp(j)>{}, fem);
                } else {
                    send(std::integral_constant<int, j>{}, pfma(omt, f[j], pmul(itc, fep)));
                    send(std::integral_constant<int, opp(j)>{}, pfma(omt, f[opp(j)], pmul(itc, fem)));
                }
            };
            pair(std::integral_constant<int, 1>{}, ux);
            pair(std::integral_constant<int, 3>{}, uy);
            pair(std::integral_constant<int, 5>{}, uz);
            pair(std::integral_constant<int, 7>{}, padd(ux, uy));
            pair(std::integral_constant<int, 9>{}, psub(ux, uy));
            pair(std::integral_constant<int, 11>{}, padd(ux, uz));
            pair(std::integral_constant<int, 13>{}, psub(ux, uz));
            pair(std::integral_constant<int, 15>{}, padd(uy, uz));
            pair(std::integral_constant<int, 17>{}, psub(uy, uz));
            // rest population: its equilibrium is rho minus the other 18
            // (equal to Eq. Equil in exact arithmetic), and in deviation
            // storage it absorbs the rounding of the 18 stored values, so
            // node mass is kept to FP32 rounding.  It stays at the node and
            // enters only the density field: it is not stored.
            const R2 q0 = padd(pfma(itc, psub(rho, fe_sum), T1 ? p2(R(0)) : pmul(omt, f[0])), resid);
            mid[0] = padd(mid[0], padd(q0, self));
            // the 18 stored values and q0 sum to rho^c: the collision
            // conserves mass
            msum = padd(msum, rho);
        }

        // x shift (all lanes take part)
#pragma unroll
        for (int q = 0; q < 5; q++) {
            R2 fromL, fromR;
            fromL.x = __shfl_up_sync(FULL, up[q].x, 1);
            fromL.y = __shfl_up_sync(FULL, up[q].y, 1);
            fromR.x = __shfl_down_sync(FULL, dn[q].x, 1);
            fromR.y = __shfl_down_sync(FULL, dn[q].y, 1);
            if (lx == 0) fromL = p2(R(0));
            if (lx == 31) fromR = p2(R(0));
            mid[q] = padd(mid[q], padd(fromL, fromR));
        }
        // values leaving the tile through x: the first lane sends left, the
        // last active lane sends right (both components at one address)
        if (active && (lx == 0 || lx == w - 1)) {
            // group q arrives at n + (x offset) + yz(q)
            const int mx = n + (lx == 0 ? oxm : oxp);
#pragma unroll
            for (int q = 0; q < 5; q++) {
                const R2 v = lx == 0 ? dn[q] : up[q];
                if (v.x != R(0) || v.y != R(0)) red_add2<R>(rnext2 + (mx + yz(q)), v.x, v.y);
            }
            if (w == 1) {  // a one-node-wide tile also sends right
#pragma unroll
                for (int q = 0; q < 5; q++)
                    if (up[q].x != R(0) || up[q].y != R(0))
                        red_add2<R>(rnext2 + (n + oxp + yz(q)), up[q].x, up[q].y);
            }
        }
        // y shift: rows exchange through shared memory; values leaving the
        // tile through y are reduced into the ring rows directly
        acc[1] = padd(acc[1], mid[0]);
        acc[2] = padd(acc[2], mid[3]);
        acc[0] = padd(acc[0], mid[4]);
#pragma unroll
        for (int q = 1; q < 9; q++) {
            if (yb_of(q) < 0) continue;
            YB2(yb_of(q), ly, lx) = mid[q];
        }
        if (active && (ly == 0 || ly == h - 1)) {
#pragma unroll
            for (int q = 1; q < 9; q++) {
                if (yb_of(q) < 0) continue;
                const int dy = grp_dy(q);
                if (!((ly == 0 && dy < 0) || (ly == h - 1 && dy > 0))) continue;
                if (mid[q].x != R(0) || mid[q].y != R(0)) red_add2<R>(rnext2 + (n + yz(q)), mid[q].x, mid[q].y);
            }
        }
        __syncthreads();

        if (active) {
#pragma unroll
            for (int q = 1; q < 9; q++) {
                if (yb_of(q) < 0) continue;
                const int dy = grp_dy(q), dz = grp_dz(q);
                const int src = ly - dy;
                if (src < 0 || src >= h) continue;
                acc[1 + dz] = padd(acc[1 + dz], YB2(yb_of(q), src, lx));
            }
            // plane z - 1 is complete: interior nodes are stored, edge and
            // ring nodes reduced
            const int pz = z - 1;
            const bool own_plane = pz >= z0;
            const bool interior = own_plane && pz <= z0 + d - 2 && pz >= z0 + 1 && lx >= 1 && lx <= w - 2 && ly >= 1 &&
                                  ly <= h - 2;
            const int m = n + ozm;
            if (interior) rnext2[m] = acc[0];
            else if (acc[0].x != R(0) || acc[0].y != R(0)) red_add2<R>(rnext2 + m, acc[0].x, acc[0].y);
            if (own_plane && !interior) rzero[m] = p2(R(0));
        }
        acc[0] = acc[1];
        acc[1] = acc[2];
        acc[2] = p2(R(0));
        // plane z + 2 replaces plane z - 1 in the window
        {
            const int t = sm_;
            sm_ = sc_;
            sc_ = sp_;
            sp_ = t;
        }

        if (more) store_window(ahead, sp_);
        rq0[0] = rq1[0];
        rq0[1] = rq1[1];
        rq1[0] = ahead.a0;
        rq1[1] = ahead.a1;

        __syncthreads();
    }
    if constexpr (StepStage<P, TY>::on) cp_async_wait_all();  // none left in flight at exit
    // last own plane and the ring plane above the chunk
    if (active) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int pz = z0 + d - 1 + k;
            const int gz = pz >= nz ? pz - nz : pz;
            const int m = nxyc + nxy * gz;
            if (acc[k].x != R(0) || acc[k].y != R(0)) red_add2<R>(rnext2 + m, acc[k].x, acc[k].y);
            if (k == 0) rzero[m] = mk2<R2>(R(0), R(0));
        }
    }

    // fluid mass produced for the next step (used by Eq. masscorr)
    {
        const unsigned FULL = 0xffffffffu;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            msum.x += __shfl_xor_sync(FULL, msum.x, off);
            msum.y += __shfl_xor_sync(FULL, msum.y, off);
        }
        if (lx == 0) {
            s_red[0][ly] = (double)msum.x;
            s_red[1][ly] = (double)msum.y;
        }
        __syncthreads();
        if (tid == 0) {
            double a0 = 0, a1 = 0;
            for (int k = 0; k < TY; k++) {
                a0 += s_red[0][k];
                a1 += s_red[1][k];
            }
            atomicAdd(&B.mass_acc[mslot * 2 + 0], a0);
            atomicAdd(&B.mass_acc[mslot * 2 + 1], a1);
        }
    }
}

}  // namespace lbp
