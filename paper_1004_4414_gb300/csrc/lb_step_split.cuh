// lb_step_split.cuh -- the fused per-step kernel of the fluid with the two
// components of a node on the two halves of a warp.
//
// Method and memory layout are those of k_step (lb_step_kernel.cuh):
// streaming with bounce-back (Eq. eqn_bounce-back), the Shan-Chen force of
// Eq. eqn_shan-chen-F with Psi of Eq. eqn_ref_dens, BGK collision towards
// the equilibrium of Eq. Equil at the common velocity u' of Sec. 2 shifted
// by tau F / rho, and the density of the next step produced by scatter, on
// the AA pattern.
//
// Difference: one thread carries one component of one node.  Lanes 0-15 of
// a warp hold the red component and lanes 16-31 the blue component of the
// same 16 nodes of an x row.  Inside a node the components meet only in
// u', which needs the partner's density and momentum: four shuffles.  A
// thread holds 18 populations instead of 36, so it needs about half the
// registers and an SM keeps twice the warps resident to hide load and store
// latency.  Tiles are 16 nodes wide.  The two components of a direction and
// node are one pair in memory, so a warp's access covers the 16 pairs of its
// nodes: 128 contiguous bytes in FP32.
#pragma once
#include "lb_step_kernel.cuh"

namespace lbp {

template <class R, int TY>
struct SplitSmem {
    static constexpr int W2 = 18, H2 = TY + 2, PLANE = W2 * H2;
    // component planes of the Psi window start 16 words apart modulo 32, so
    // that the two half-warps, which read the same position of different
    // components, hit different banks
    static constexpr int CS = PLANE + ((16 - PLANE % 32) + 32) % 32;
    static constexpr size_t psi_elems = (size_t)3 * 2 * CS;
    static constexpr size_t yb_elems = (size_t)6 * TY * 32;
    static constexpr size_t bytes = (psi_elems + yb_elems) * sizeof(R) + (size_t)3 * PLANE + 64;
};

// Block shape 32 x TY; a CTA owns a tile of 16 x TY nodes and marches through
// d planes.  Register budget: 32 resident warps per SM.
template <class P, int PAR, int TY, bool T1, bool BB>
static __global__ void __launch_bounds__(32 * TY, 32 / TY)
    k_step_split(const BoxDev* __restrict__ boxes, const TileDev* __restrict__ tiles, Shared sh, int rc, int rn,
                 int rz, int mslot) {
    using R = typename P::real;
    using S = typename P::st;
    using SM = SplitSmem<R, TY>;
    constexpr int W2 = SM::W2, CS = SM::CS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* s_psi = reinterpret_cast<R*>(smem_raw);                         // [3 slots][2][CS]
    R* s_yb = s_psi + SM::psi_elems;                                   // [6][TY][32 lanes]
    uint8_t* s_flg = reinterpret_cast<uint8_t*>(s_yb + SM::yb_elems);  // [3 slots][H2][W2]
    __shared__ double s_red[2][TY];

    const TileDev T = tiles[blockIdx.x];
    const BoxDev& B = boxes[T.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = B.N;
    const int nxy = nx * ny;
    // density ring: component c of node m at [2 m + c]
    const R* __restrict__ rcur = reinterpret_cast<const R*>(B.rho[rc]);
    R* __restrict__ rnext = reinterpret_cast<R*>(B.rho[rn]);
    R* __restrict__ rzero = reinterpret_cast<R*>(B.rho[rz]);
    const uint8_t* __restrict__ gflags = B.flags;
    const Pop<P> pop(B);
    const R rho0 = (R)B.rho0, irho0 = R(1) / (R)B.rho0, g = (R)B.g;
    const R itau0 = (R)B.inv_tau[0], itau1 = (R)B.inv_tau[1];
    R* const rnext_c = rnext + (threadIdx.x >> 4);  // this thread's component: node m at rnext_c[2 m]
    const R wax = (R)B.scw_axis, wdg = (R)B.scw_diag;
    const R bfx = (R)B.body[0], bfy = (R)B.body[1], bfz = (R)B.body[2];
    const int velmode = B.vel_mode;

    const int lane = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lane;
    const int c = lane >> 4, lx = lane & 15;  // component, column in the tile
    const R tauc = (R)B.tau[c], itauc = (R)B.inv_tau[c];
    // this component's population arrays and deviation constants
    S* const cbase = pop.at(c, P::dev ? 1 : 0, 0);
    const size_t dstride = 2 * pop.N;  // elements between direction arrays
    float zra = 0.f, zrd = 0.f, refc = 0.f;
    if constexpr (P::dev) {
        zra = c ? pop.zr[1][0] : pop.zr[0][0];
        zrd = c ? pop.zr[1][1] : pop.zr[0][1];
        refc = (float)(c ? pop.ref[1] : pop.ref[0]);
    }
    // this component of direction i >= 1 at node m
    auto dirp = [&](int i, int m) -> S* { return cbase + (size_t)(P::dev ? i - 1 : i) * dstride + 2 * (size_t)m; };
    auto ldv = [&](const S* p, int i) -> R {
        if constexpr (P::dev) return fmaf(wgt<float>(i), to_f(*p), is_axis(i) ? zra : zrd);
        else return *p;
    };
    // stores v, returns the value the next load will see
    auto stv = [&](S* p, int i, R v) -> R {
        if constexpr (P::dev) {
            const S q = from_f<S>(fmaf(v, 1.0f / wgt<float>(i), -refc));
            *p = q;
            return fmaf(wgt<float>(i), to_f(q), is_axis(i) ? zra : zrd);
        } else {
            *p = v;
            return v;
        }
    };

    const int w = T.w, h = T.h, d = T.d, x0 = T.x0, y0 = T.y0, z0 = T.z0;
    const bool active = lx < w && ly < h;
    const int x = active ? x0 + lx : x0, y = active ? y0 + ly : y0;
    const int oxm = (x == 0) ? nx - 1 : -1, oxp = (x == nx - 1) ? -(nx - 1) : 1;
    const int oym = (y == 0) ? (ny - 1) * nx : -nx, oyp = (y == ny - 1) ? -(ny - 1) * nx : nx;
    const int nxyc = x + nx * y;

    auto PSI = [&](int s, int cc, int r, int k) -> R& { return s_psi[(s * 2 + cc) * CS + r * W2 + k]; };
    auto FLG = [&](int s, int r, int k) -> uint8_t& { return s_flg[(s * SM::H2 + r) * W2 + k]; };
    auto YB = [&](int q, int r) -> R& { return s_yb[(q * TY + r) * 32 + lane]; };

    // window ring: thread tid < nring takes ring node (ring_r, ring_k), both
    // components
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
    struct WinRaw {
        R a, b0, b1;
        uint8_t af, bf;
    };
    auto fetch_window = [&](int zz) {
        WinRaw v{R(0), R(0), R(0), 0, 0};
        const int gz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        const int pb = nxy * gz;
        if (active) {
            const int n = pb + nxyc;
            v.a = rcur[2 * (size_t)n + c];
            if (c == 0) v.af = gflags[n];
        }
        if (tid < nring) {
            const int n = pb + ring_xy;
            v.b0 = rcur[2 * (size_t)n];
            v.b1 = rcur[2 * (size_t)n + 1];
            v.bf = gflags[n];
        }
        return v;
    };
    auto store_window = [&](const WinRaw& v, int s) {
        if (active) {
            PSI(s, c, ly + 1, lx + 1) = psi_of<R>(v.a, rho0, irho0);
            if (c == 0) FLG(s, ly + 1, lx + 1) = v.af;
        }
        if (tid < nring) {
            PSI(s, 0, ring_r, ring_k) = psi_of<R>(v.b0, rho0, irho0);
            PSI(s, 1, ring_r, ring_k) = psi_of<R>(v.b1, rho0, irho0);
            FLG(s, ring_r, ring_k) = v.bf;
        }
    };

    int sm_ = 0, sc_ = 1, sp_ = 2;
    store_window(fetch_window(z0 - 1), sm_);
    // this component's density at the own node of planes z and z + 1: the
    // window fetches it anyway, and it is the node's rho^c
    R rq0, rq1;
    {
        const WinRaw v0 = fetch_window(z0);
        store_window(v0, sc_);
        rq0 = v0.a;
        const WinRaw v1 = fetch_window(z0 + 1);
        store_window(v1, sp_);
        rq1 = v1.a;
    }
    R acc[3] = {R(0), R(0), R(0)};  // own-column partial densities of planes z-1, z, z+1
    R msum = R(0);
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    for (int z = z0; z < z0 + d; z++) {
        const bool more = z + 1 < z0 + d;
        WinRaw ahead{R(0), R(0), R(0), 0, 0};
        if (more) ahead = fetch_window(z + 2);
        const int ozm = (z == 0) ? (nz - 1) * nxy : -nxy, ozp = (z == nz - 1) ? -(nz - 1) * nxy : nxy;
        const int n = nxyc + nxy * z;
        auto off = [&](int i) -> int {
            return (cx(i) < 0 ? oxm : (cx(i) > 0 ? oxp : 0)) + (cy(i) < 0 ? oym : (cy(i) > 0 ? oyp : 0)) +
                   (cz(i) < 0 ? ozm : (cz(i) > 0 ? ozp : 0));
        };
        auto slot_dz = [&](int dz) { return dz < 0 ? sm_ : (dz > 0 ? sp_ : sc_); };
        // offset of the node (x, y + dy, z + dz) of scatter group q
        auto yz = [&](int q) -> int {
            const int dy = grp_dy(q), dz = grp_dz(q);
            return (dy < 0 ? oym : (dy > 0 ? oyp : 0)) + (dz < 0 ? ozm : (dz > 0 ? ozp : 0));
        };

        const uint8_t fl = active ? FLG(sc_, ly + 1, lx + 1) : FL_SOLID;
        const bool fluid = active && !(fl & FL_SOLID);
        unsigned smask = 0;
        R f[19];
        R rho = R(1), jx = R(0), jy = R(0), jz = R(0), Fx = R(0), Fy = R(0), Fz = R(0);
        if (fluid) {
            if constexpr (BB) {
#pragma unroll
                for (int i = 1; i < 19; i++)
                    smask |= (unsigned)(FLG(slot_dz(cz(i)), ly + 1 + cy(i), lx + 1 + cx(i)) & FL_SOLID) << i;
            }
#pragma unroll
            for (int i = 1; i < 19; i++) {
                const S* p = PAR == 0 ? dirp(i, n) : dirp(opp(i), n + off(opp(i)));
                f[i] = ldv(p, i);
            }
            // rho^c is the density field (the sum of the values the previous
            // step sent here); the rest population is rho^c minus the 18
            // moving ones and is needed only for tau != 1
            R r = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
            for (int i = 1; i < 19; i++) {
                if constexpr (!T1) r += f[i];
                if (cx(i) > 0) ax += f[i];
                if (cx(i) < 0) ax -= f[i];
                if (cy(i) > 0) ay += f[i];
                if (cy(i) < 0) ay -= f[i];
                if (cz(i) > 0) az += f[i];
                if (cz(i) < 0) az -= f[i];
            }
            rho = rq0;
            f[0] = T1 ? R(0) : rq0 - r;
            jx = ax;
            jy = ay;
            jz = az;
            const int cb = 1 - c;
            R sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int i = 1; i < 19; i++) {
                const R p = (is_axis(i) ? wax : wdg) * PSI(slot_dz(cz(i)), cb, ly + 1 + cy(i), lx + 1 + cx(i));
                if (cx(i) > 0) sx += p;
                if (cx(i) < 0) sx -= p;
                if (cy(i) > 0) sy += p;
                if (cy(i) < 0) sy -= p;
                if (cz(i) > 0) sz += p;
                if (cz(i) < 0) sz -= p;
            }
            const R pc = -g * PSI(sc_, c, ly + 1, lx + 1);
            Fx = pc * sx + rho * bfx;
            Fy = pc * sy + rho * bfy;
            Fz = pc * sz + rho * bfz;
        }
        // the partner component of the same node (all lanes take part)
        const R rho_o = __shfl_xor_sync(FULL, rho, 16);
        const R jx_o = __shfl_xor_sync(FULL, jx, 16);
        const R jy_o = __shfl_xor_sync(FULL, jy, 16);
        const R jz_o = __shfl_xor_sync(FULL, jz, 16);
        R ux = R(0), uy = R(0), uz = R(0);
        if (fluid) {
            const R r0 = c ? rho_o : rho, r1 = c ? rho : rho_o;
            const R iden = R(1) / (r0 * itau0 + r1 * itau1);
            const R ir = R(1) / rho;
            R bx_, by_, bz_;
            if (velmode) {
                bx_ = jx * ir;
                by_ = jy * ir;
                bz_ = jz * ir;
            } else {
                const R x0_ = c ? jx_o : jx, x1_ = c ? jx : jx_o;
                const R y0_ = c ? jy_o : jy, y1_ = c ? jy : jy_o;
                const R z0_ = c ? jz_o : jz, z1_ = c ? jz : jz_o;
                bx_ = (x0_ * itau0 + x1_ * itau1) * iden;
                by_ = (y0_ * itau0 + y1_ * itau1) * iden;
                bz_ = (z0_ * itau0 + z1_ * itau1) * iden;
            }
            ux = bx_ + tauc * Fx * ir;
            uy = by_ + tauc * Fy * ir;
            uz = bz_ + tauc * Fz * ir;
            if (c == 0) {
                const R rt = rho + rho_o;
                const R vx = jx + jx_o, vy = jy + jy_o, vz = jz + jz_o;
                if (!(rho > R(0)) || !(rho_o > R(0)) || !(vx * vx + vy * vy + vz * vz < R(0.25) * rt * rt))
                    set_err(sh.err, ERR_UNSTABLE);
            }
        }

        R mid[9], up[5], dn[5];
#pragma unroll
        for (int q = 0; q < 9; q++) mid[q] = R(0);
#pragma unroll
        for (int q = 0; q < 5; q++) up[q] = dn[q] = R(0);
        if (fluid) {
            const R itc = T1 ? R(1) : itauc;
            const R omt = T1 ? R(0) : R(1) - itc;
            const R uu = ux * ux + uy * uy + uz * uz;
            const R a0 = R(1) - R(1.5) * uu;
            const R rw1 = rho * wgt<R>(1), rw7 = rho * wgt<R>(7);
            R resid = R(0), fe_sum = R(0), self = R(0);
            // stores as in k_step: target fluid -> even steps slot opp(j) of
            // x, odd steps slot j of y; target solid -> even steps slot j of
            // y, odd steps slot opp(j) of x
            auto send = [&](auto JC, R fs) {
                constexpr int j = decltype(JC)::value;
                const bool solid = BB && ((smask >> j) & 1u);
                S* p;
                if (PAR == 0) p = solid ? dirp(j, n + off(j)) : dirp(opp(j), n);
                else p = solid ? dirp(opp(j), n) : dirp(j, n + off(j));
                const R q = stv(p, j, fs);
                if constexpr (P::dev) resid += fs - q;
                const R qf = solid ? R(0) : q;
                self += solid ? q : R(0);
                constexpr int gq = grp_of(j);
                if (cx(j) == 0) mid[gq] += qf;
                else if (cx(j) > 0) up[gq] += qf;
                else dn[gq] += qf;
            };
            auto pair = [&](auto JC, R cu) {
                constexpr int j = decltype(JC)::value;
                const R rw = is_axis(j) ? rw1 : rw7;
                const R cu2 = cu * cu;
                const R E = a0 + R(4.5) * cu2;
                const R O = cu * (R(3) + R(4.5) * cu2 - R(4.5) * uu);
                const R fep = rw * (E + O), fem = rw * (E - O);
                fe_sum += fep + fem;
                if constexpr (T1) {
                    send(std::integral_constant<int, j>{}, fep);
                    send(std::integral_constant<int, opp(j)>{}, fem);
                } else {
                    send(std::integral_constant<int, j>{}, omt * f[j] + itc * fep);
                    send(std::integral_constant<int, opp(j)>{}, omt * f[opp(j)] + itc * fem);
                }
            };
            pair(std::integral_constant<int, 1>{}, ux);
            pair(std::integral_constant<int, 3>{}, uy);
            pair(std::integral_constant<int, 5>{}, uz);
            pair(std::integral_constant<int, 7>{}, ux + uy);
            pair(std::integral_constant<int, 9>{}, ux - uy);
            pair(std::integral_constant<int, 11>{}, ux + uz);
            pair(std::integral_constant<int, 13>{}, ux - uz);
            pair(std::integral_constant<int, 15>{}, uy + uz);
            pair(std::integral_constant<int, 17>{}, uy - uz);
            // the rest population stays at the node; it is not stored
            const R q0 = (T1 ? R(0) : omt * f[0]) + itc * (rho - fe_sum) + resid;
            mid[0] += q0 + self;
            msum += rho;
        }
        // x shift inside each half-warp
#pragma unroll
        for (int q = 0; q < 5; q++) {
            R fromL = __shfl_up_sync(FULL, up[q], 1, 16);
            R fromR = __shfl_down_sync(FULL, dn[q], 1, 16);
            if (lx == 0) fromL = R(0);
            if (lx == 15) fromR = R(0);
            mid[q] += fromL + fromR;
        }
        if (active && (lx == 0 || lx == w - 1)) {
            const int mx = n + (lx == 0 ? oxm : oxp);
#pragma unroll
            for (int q = 0; q < 5; q++) {
                const R v = lx == 0 ? dn[q] : up[q];
                if (v != R(0)) red_add(rnext_c + 2 * (size_t)(mx + yz(q)), v);
            }
            if (w == 1) {  // a one-node-wide tile also sends right
#pragma unroll
                for (int q = 0; q < 5; q++)
                    if (up[q] != R(0)) red_add(rnext_c + 2 * (size_t)(n + oxp + yz(q)), up[q]);
            }
        }
        acc[1] += mid[0];
        acc[2] += mid[3];
        acc[0] += mid[4];
#pragma unroll
        for (int q = 1; q < 9; q++) {
            if (yb_of(q) < 0) continue;
            YB(yb_of(q), ly) = mid[q];
        }
        if (active && (ly == 0 || ly == h - 1)) {
#pragma unroll
            for (int q = 1; q < 9; q++) {
                if (yb_of(q) < 0) continue;
                const int dy = grp_dy(q);
                if (!((ly == 0 && dy < 0) || (ly == h - 1 && dy > 0))) continue;
                if (mid[q] != R(0)) red_add(rnext_c + 2 * (size_t)(n + yz(q)), mid[q]);
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
                acc[1 + dz] += YB(yb_of(q), src);
            }
            // plane z - 1 is complete
            const int pz = z - 1;
            const bool own_plane = pz >= z0;
            const bool interior = own_plane && pz <= z0 + d - 2 && pz >= z0 + 1 && lx >= 1 && lx <= w - 2 && ly >= 1 &&
                                  ly <= h - 2;
            const int m = n + ozm;
            if (interior) rnext_c[2 * (size_t)m] = acc[0];
            else if (acc[0] != R(0)) red_add(rnext_c + 2 * (size_t)m, acc[0]);
            if (own_plane && !interior) rzero[2 * (size_t)m + c] = R(0);
        }
        acc[0] = acc[1];
        acc[1] = acc[2];
        acc[2] = R(0);
        {
            const int t = sm_;
            sm_ = sc_;
            sc_ = sp_;
            sp_ = t;
        }
        if (more) store_window(ahead, sp_);
        rq0 = rq1;
        rq1 = ahead.a;
        __syncthreads();
    }
    if (active) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int pz = z0 + d - 1 + k;
            const int gz = pz >= nz ? pz - nz : pz;
            const int m = nxyc + nxy * gz;
            if (acc[k] != R(0)) red_add(rnext_c + 2 * (size_t)m, acc[k]);
            if (k == 0) rzero[2 * (size_t)m + c] = R(0);
        }
    }

    // fluid mass produced for the next step (used by Eq. masscorr): sum over
    // each half-warp, then over the rows
    {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) msum += __shfl_xor_sync(FULL, msum, o);
        if (lx == 0) s_red[c][ly] = (double)msum;
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
