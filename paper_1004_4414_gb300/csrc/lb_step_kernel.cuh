// lb_step_kernel.cuh -- the fused per-step kernel of the fluid: streaming,
// moving-wall bounce-back with momentum exchange, Shan-Chen force,
// cubic-equilibrium BGK collision, the shell Shan-Chen force on the
// particles, and the density field of the next step.
//
// Method (paper): Eq. eq:boltz with the BGK operator and the equilibrium of
// Eq. Equil at the velocity shifted by tau F / rho (Sec. II); the force of
// Eq. eqn_shan-chen-F with Psi of Eq. eqn_ref_dens over the 18 D3Q19 links;
// bounce-back with the moving-wall term and the momentum-exchange force
// (Eqs. eqn_bounce-back, eqn_ladd_bewegtewand; coefficient 6 zeta_j =
// 2 zeta_j / c_s^2); the force of the virtual fluid on its particle
// (Eq. eqn_shan_chen_particle).
//
// GB300 design:
//   * Populations are kept in place with the AA pattern: on even steps a node
//     reads its own 19 slots and writes the post-collision values to the
//     opposite slots of itself; on odd steps it reads f_i from slot opp(i) of
//     x - c_i and writes f*_j to slot j of x + c_j.  A population whose
//     stream target is solid is reflected into slot opp(j) of the node on
//     both parities, which is exactly where the next step reads it.  Memory
//     per population is one slot; every slot is read once and written once
//     per step.
//   * A CTA owns a column tile of 32 x TY nodes (one warp per x row, so all
//     global traffic is coalesced along x) and marches through a chunk of z
//     planes.  Psi and the node flags of the tile plus a one-node ring are
//     staged in a three-plane shared-memory ring buffer, so each density
//     value is loaded from HBM/L2 once per tile.
//   * The Shan-Chen force needs Psi of all neighbours at the same time
//     level.  Instead of a second pass over the populations, the kernel
//     produces rho(t+1) itself: each post-streaming value is added (shared
//     memory atomics) to a three-plane accumulator at its destination node.
//     Nodes whose whole stencil lies inside the tile are written with plain
//     stores; tile-edge and ring nodes are added with global atomics into a
//     density field that was zeroed at those nodes during the previous step
//     (ring of three density buffers: current, next, to-zero).
//   * Particle forces are summed per node (all reflected links of a node
//     give forces parallel to c_j, so the torque of the node is
//     (x - X_p) x F), reduced across the warp per particle with shuffles,
//     and added to FP64 accumulators with one atomic per (warp, particle).
#pragma once
#include "lb_common.cuh"

namespace lbp {

// Sum (F, T) of the lanes that share a particle key, one FP64 atomic per
// distinct key in the warp.  All 32 lanes of the warp must call it.
__device__ __forceinline__ void warp_particle_add(int key, const double v[6], double* force) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(FULL, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(FULL, key, leader);
        const bool mine = (key == k);
        const unsigned grp = __ballot_sync(FULL, mine);
        double s[6];
#pragma unroll
        for (int a = 0; a < 6; a++) s[a] = mine ? v[a] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int a = 0; a < 6; a++) s[a] += __shfl_xor_sync(FULL, s[a], off);
        if (lane == leader)
#pragma unroll
            for (int a = 0; a < 6; a++) atomicAdd(&force[(size_t)k * 6 + a], s[a]);
        pending &= ~grp;
    }
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

template <class R>
__device__ __forceinline__ R psi_of(R rho, R rho0) {
    if constexpr (sizeof(R) == 8) return rho0 * (1.0 - exp(-rho / rho0));
    else return rho0 * (1.0f - expf(-rho / rho0));
}

// shared memory of one CTA, in elements of R
template <class R, int TY>
struct StepSmem {
    static constexpr int W2 = 34, H2 = TY + 2, PLANE = W2 * H2;
    static constexpr size_t bytes = (size_t)2 * 3 * 2 * PLANE * sizeof(R) + (size_t)3 * PLANE + 64;
};

template <class P, int PAR, int TY>
static __global__ void __launch_bounds__(32 * TY)
    k_step(const BoxDev* __restrict__ boxes, const TileDev* __restrict__ tiles, Shared sh, int rc, int rn, int rz,
           int mslot) {
    using R = typename P::real;
    using SM = StepSmem<R, TY>;
    constexpr int W2 = SM::W2, H2 = SM::H2, PLANE = SM::PLANE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* s_psi = reinterpret_cast<R*>(smem_raw);    // [3 slots][2 comps][H2][W2]
    R* s_acc = s_psi + 3 * 2 * PLANE;             // [3 slots][2 comps][H2][W2]
    uint8_t* s_flg = reinterpret_cast<uint8_t*>(s_acc + 3 * 2 * PLANE);  // [3 slots][H2][W2]
    __shared__ double s_red[2][32];

    const TileDev T = tiles[blockIdx.x];
    const BoxDev& B = boxes[T.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = B.N;
    const R* __restrict__ rcur = reinterpret_cast<const R*>(B.rho[rc]);
    R* __restrict__ rnext = reinterpret_cast<R*>(B.rho[rn]);
    R* __restrict__ rzero = reinterpret_cast<R*>(B.rho[rz]);
    const uint8_t* __restrict__ gflags = B.flags;
    const int32_t* __restrict__ gowner = B.owner;
    const Pop<P> pop(B);
    const R rho0 = (R)B.rho0, g = (R)B.g;
    const R tau0 = (R)B.tau[0], tau1 = (R)B.tau[1], itau0 = (R)B.inv_tau[0], itau1 = (R)B.inv_tau[1];
    const R wax = (R)B.scw_axis, wdg = (R)B.scw_diag;
    const R bx = (R)B.body[0], by = (R)B.body[1], bz = (R)B.body[2];
    const int velmode = B.vel_mode;

    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * 32 + lx;
    constexpr int NTHR = 32 * TY;
    const int w = T.w, h = T.h, d = T.d, x0 = T.x0, y0 = T.y0, z0 = T.z0;
    const bool active = lx < w && ly < h;
    const int x = x0 + lx, y = y0 + ly;
    // wrapped neighbour coordinates (index 1 + offset)
    const int xw[3] = {x == 0 ? nx - 1 : x - 1, x, x + 1 >= nx ? x + 1 - nx : x + 1};
    const int yw[3] = {y == 0 ? ny - 1 : y - 1, y, y + 1 >= ny ? y + 1 - ny : y + 1};

    auto slot = [&](int zz) { return (zz - z0 + 1) % 3; };
    auto PSI = [&](int s, int c, int r, int k) -> R& { return s_psi[((s * 2 + c) * H2 + r) * W2 + k]; };
    auto ACC = [&](int s, int c, int r, int k) -> R& { return s_acc[((s * 2 + c) * H2 + r) * W2 + k]; };
    auto FLG = [&](int s, int r, int k) -> uint8_t { return s_flg[(s * H2 + r) * W2 + k]; };

    auto load_plane = [&](int zz) {
        const int s = slot(zz), gz = wrapi(zz, nz);
        const int cnt = (h + 2) * (w + 2);
        for (int idx = tid; idx < cnt; idx += NTHR) {
            const int r = idx / (w + 2), k = idx - r * (w + 2);
            const int gx = wrapi(x0 + k - 1, nx), gy = wrapi(y0 + r - 1, ny);
            const int n = gx + nx * (gy + ny * gz);
            PSI(s, 0, r, k) = psi_of<R>(rcur[n], rho0);
            PSI(s, 1, r, k) = psi_of<R>(rcur[N + n], rho0);
            s_flg[(s * H2 + r) * W2 + k] = gflags[n];
        }
        for (int idx = tid; idx < 2 * PLANE; idx += NTHR) s_acc[s * 2 * PLANE + idx] = R(0);
    };

    auto flush_plane = [&](int pz) {
        const int s = slot(pz), gz = wrapi(pz, nz);
        const bool own_plane = pz >= z0 && pz < z0 + d;
        const bool int_plane = pz >= z0 + 1 && pz <= z0 + d - 2;
        const int cnt = (h + 2) * (w + 2);
        for (int idx = tid; idx < cnt; idx += NTHR) {
            const int r = idx / (w + 2), k = idx - r * (w + 2);
            const int lxp = k - 1, lyp = r - 1;
            const bool own = own_plane && lxp >= 0 && lxp < w && lyp >= 0 && lyp < h;
            const bool interior = int_plane && lxp >= 1 && lxp <= w - 2 && lyp >= 1 && lyp <= h - 2;
            const int n = wrapi(x0 + lxp, nx) + nx * (wrapi(y0 + lyp, ny) + ny * gz);
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const R v = ACC(s, c, r, k);
                if (interior) rnext[(size_t)c * N + n] = v;
                else if (v != R(0)) atomicAdd(&rnext[(size_t)c * N + n], v);
            }
            if (own && !interior) {
                rzero[n] = R(0);
                rzero[(size_t)N + n] = R(0);
            }
        }
    };

    double msum0 = 0.0, msum1 = 0.0;
    load_plane(z0 - 1);
    load_plane(z0);

    for (int z = z0; z < z0 + d; z++) {
        load_plane(z + 1);
        __syncthreads();

        int pkey = -1;
        double pv[6] = {0, 0, 0, 0, 0, 0};
        if (active) {
            const int zc = wrapi(z, nz);
            const int zw[3] = {zc == 0 ? nz - 1 : zc - 1, zc, zc + 1 >= nz ? zc + 1 - nz : zc + 1};
            const int sl[3] = {slot(z - 1), slot(z), slot(z + 1)};
            auto nidx = [&](int dx, int dy, int dz) { return xw[1 + dx] + nx * (yw[1 + dy] + ny * zw[1 + dz]); };
            const int n = nidx(0, 0, 0);
            const uint8_t fl = FLG(sl[1], ly + 1, lx + 1);

            // Shan-Chen force sums S^c = sum_i W_i Psi^cbar(x + c_i) c_i
            auto sc_sum = [&](int cb, R& sx, R& sy, R& sz) {
                sx = sy = sz = R(0);
#pragma unroll
                for (int i = 1; i < 19; i++) {
                    const R wl = is_axis(i) ? wax : wdg;
                    const R p = PSI(sl[1 + cz(i)], cb, ly + 1 + cy(i), lx + 1 + cx(i));
                    sx += wl * p * R(cx(i));
                    sy += wl * p * R(cy(i));
                    sz += wl * p * R(cz(i));
                }
            };

            if (!(fl & FL_SOLID)) {
                // ---------------------------------------------- fluid node
                R f[2][19];
#pragma unroll
                for (int c = 0; c < 2; c++)
#pragma unroll
                    for (int i = 0; i < 19; i++) {
                        if (PAR == 0 || i == 0) {
                            f[c][i] = pop.load(c, i, n);
                        } else {
                            const bool src_solid = FLG(sl[1 - cz(i)], ly + 1 - cy(i), lx + 1 - cx(i)) & FL_SOLID;
                            f[c][i] = src_solid ? pop.load(c, i, n) : pop.load(c, opp(i), nidx(-cx(i), -cy(i), -cz(i)));
                        }
                    }
                R rho[2], jx[2], jy[2], jz[2];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    R r = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
                    for (int i = 0; i < 19; i++) {
                        r += f[c][i];
                        ax += R(cx(i)) * f[c][i];
                        ay += R(cy(i)) * f[c][i];
                        az += R(cz(i)) * f[c][i];
                    }
                    rho[c] = r;
                    jx[c] = ax;
                    jy[c] = ay;
                    jz[c] = az;
                }
                R Fx[2], Fy[2], Fz[2];
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    R sx, sy, sz;
                    sc_sum(1 - c, sx, sy, sz);
                    const R pc = PSI(sl[1], c, ly + 1, lx + 1);
                    Fx[c] = -g * pc * sx + rho[c] * bx;
                    Fy[c] = -g * pc * sy + rho[c] * by;
                    Fz[c] = -g * pc * sz + rho[c] * bz;
                }
                R ux[2], uy[2], uz[2];
                {
                    const R den = rho[0] * itau0 + rho[1] * itau1;
                    const R upx = (jx[0] * itau0 + jx[1] * itau1) / den;
                    const R upy = (jy[0] * itau0 + jy[1] * itau1) / den;
                    const R upz = (jz[0] * itau0 + jz[1] * itau1) / den;
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        const R tc = c == 0 ? tau0 : tau1;
                        const R ir = R(1) / rho[c];
                        const R basex = velmode ? jx[c] * ir : upx;
                        const R basey = velmode ? jy[c] * ir : upy;
                        const R basez = velmode ? jz[c] * ir : upz;
                        ux[c] = basex + tc * Fx[c] * ir;
                        uy[c] = basey + tc * Fy[c] * ir;
                        uz[c] = basez + tc * Fz[c] * ir;
                    }
                    const R rt = rho[0] + rho[1];
                    const R vx = (jx[0] + jx[1]) / rt, vy = (jy[0] + jy[1]) / rt, vz = (jz[0] + jz[1]) / rt;
                    const R v2 = vx * vx + vy * vy + vz * vz;
                    if (!(rho[0] > R(0)) || !(rho[1] > R(0)) || !(v2 < R(0.25))) set_err(sh.err, ERR_UNSTABLE);
                }

                // cached data of the last particle seen on a reflected link
                int cp = -1;
                double cX[3] = {0, 0, 0}, cU[3] = {0, 0, 0}, cW[3] = {0, 0, 0};
                double nF[3] = {0, 0, 0};
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    const R itc = c == 0 ? itau0 : itau1;
                    const R uu = ux[c] * ux[c] + uy[c] * uy[c] + uz[c] * uz[c];
                    R resid = R(0);
                    R sent = R(0);
#pragma unroll
                    for (int j = 1; j < 19; j++) {
                        const R cuj = R(cx(j)) * ux[c] + R(cy(j)) * uy[c] + R(cz(j)) * uz[c];
                        const R fe = wgt<R>(j) * rho[c] *
                                     (R(1) + R(3) * cuj + R(4.5) * cuj * cuj - R(1.5) * uu +
                                      R(4.5) * cuj * cuj * cuj - R(4.5) * uu * cuj);
                        const R fs = f[c][j] - (f[c][j] - fe) * itc;
                        const uint8_t dfl = FLG(sl[1 + cz(j)], ly + 1 + cy(j), lx + 1 + cx(j));
                        if (!(dfl & FL_SOLID)) {
                            const R q = (PAR == 0) ? pop.store(c, opp(j), n, fs)
                                                   : pop.store(c, j, nidx(cx(j), cy(j), cz(j)), fs);
                            atomicAdd(&ACC(sl[1 + cz(j)], c, ly + 1 + cy(j), lx + 1 + cx(j)), q);
                            resid += fs - q;
                            sent += q;
                        } else {
                            const int p = gowner[nidx(cx(j), cy(j), cz(j))];
                            R cu = R(0);
                            double r[3];
                            if (p >= 0) {
                                if (p != cp) {
                                    const PartState ps = sh.part[p];
#pragma unroll
                                    for (int a = 0; a < 3; a++) {
                                        cX[a] = ps.X[a];
                                        cU[a] = ps.U[a];
                                        cW[a] = ps.W[a];
                                    }
                                    cp = p;
                                }
                                // surface velocity at the link midpoint x + c_j / 2
                                r[0] = mimg((double)x + 0.5 * cx(j) - cX[0], (double)nx);
                                r[1] = mimg((double)y + 0.5 * cy(j) - cX[1], (double)ny);
                                r[2] = mimg((double)zc + 0.5 * cz(j) - cX[2], (double)nz);
                                const double usx = cU[0] + cW[1] * r[2] - cW[2] * r[1];
                                const double usy = cU[1] + cW[2] * r[0] - cW[0] * r[2];
                                const double usz = cU[2] + cW[0] * r[1] - cW[1] * r[0];
                                cu = (R)(usx * cx(j) + usy * cy(j) + usz * cz(j));
                            }
                            const R wall = R(6) * wgt<R>(j) * rho[c] * cu;
                            const R b = fs - wall;
                            const R q = pop.store(c, opp(j), n, b);
                            atomicAdd(&ACC(sl[1], c, ly + 1, lx + 1), q);
                            resid += b - q;
                            sent += q;
                            if (p >= 0) {
                                const double mag = 2.0 * (double)fs - (double)wall;
                                const double lf[3] = {mag * cx(j), mag * cy(j), mag * cz(j)};
                                if (pkey < 0 || pkey == p) {
                                    pkey = p;
#pragma unroll
                                    for (int a = 0; a < 3; a++) nF[a] += lf[a];
                                } else {
                                    // a second particle on this node's links: add directly
                                    double tq[3];
                                    cross3(r, lf, tq);
                                    for (int a = 0; a < 3; a++) {
                                        atomicAdd(&sh.force[(size_t)p * 6 + a], lf[a]);
                                        atomicAdd(&sh.force[(size_t)p * 6 + 3 + a], tq[a]);
                                    }
                                }
                            }
                        }
                    }
                    // rest population; in deviation storage it absorbs the
                    // rounding of the 18 stored values so node mass is exact
                    const R fe0 = wgt<R>(0) * rho[c] * (R(1) - R(1.5) * uu);
                    const R fs0 = f[c][0] - (f[c][0] - fe0) * itc + resid;
                    const R q0 = pop.store(c, 0, n, fs0);
                    atomicAdd(&ACC(sl[1], c, ly + 1, lx + 1), q0);
                    sent += q0;
                    if (c == 0) msum0 += (double)sent;
                    else msum1 += (double)sent;
                }
                if (pkey >= 0) {
                    const PartState ps = sh.part[pkey];
                    const double rr[3] = {mimg((double)x - ps.X[0], (double)nx), mimg((double)y - ps.X[1], (double)ny),
                                          mimg((double)zc - ps.X[2], (double)nz)};
                    double tq[3];
                    cross3(rr, nF, tq);
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        pv[a] = nF[a];
                        pv[3 + a] = tq[a];
                    }
                }
            } else if (fl & FL_SHELL) {
                // ---------------------------------- shell node: virtual fluid
                const int p = gowner[n];
                if (p >= 0) {
                    double Ft[3] = {0, 0, 0};
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        R sx, sy, sz;
                        sc_sum(1 - c, sx, sy, sz);
                        const R pc = PSI(sl[1], c, ly + 1, lx + 1);
                        Ft[0] += (double)(-g * pc * sx);
                        Ft[1] += (double)(-g * pc * sy);
                        Ft[2] += (double)(-g * pc * sz);
                    }
                    const PartState ps = sh.part[p];
                    const double rr[3] = {mimg((double)x - ps.X[0], (double)nx), mimg((double)y - ps.X[1], (double)ny),
                                          mimg((double)zc - ps.X[2], (double)nz)};
                    double tq[3];
                    cross3(rr, Ft, tq);
                    pkey = p;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        pv[a] = Ft[a];
                        pv[3 + a] = tq[a];
                    }
                }
            }
        }
        warp_particle_add(pkey, pv, sh.force);
        __syncthreads();
        flush_plane(z - 1);
        __syncthreads();
    }
    flush_plane(z0 + d - 1);
    flush_plane(z0 + d);

    // fluid mass produced for the next step (used by Eq. masscorr)
    {
        const unsigned FULL = 0xffffffffu;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            msum0 += __shfl_xor_sync(FULL, msum0, off);
            msum1 += __shfl_xor_sync(FULL, msum1, off);
        }
        if (lx == 0) {
            s_red[0][ly] = msum0;
            s_red[1][ly] = msum1;
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
