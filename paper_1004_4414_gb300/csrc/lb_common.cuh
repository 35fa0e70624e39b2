// lb_common.cuh -- shared device definitions of the sm_103a library:
// D3Q19 lattice, box and tile descriptors, population storage policies,
// SplitMix64 and the cubic equilibrium.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbp {

// ---------------------------------------------------------------- lattice
// D3Q19 (Sec. II): rest, 6 axis links, 12 face diagonals in opposite pairs
// (odd i, i + 1).  The order is the library's canonical export order.
__host__ __device__ constexpr int cx(int i) {
    constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr bool is_axis(int i) { return i >= 1 && i <= 6; }
// lattice weights zeta_i: 1/3, 1/18 (axis), 1/36 (diagonal)
template <class R>
__host__ __device__ constexpr R wgt(int i) {
    return i == 0 ? R(1) / R(3) : (i <= 6 ? R(1) / R(18) : R(1) / R(36));
}

// flag bits of a node
constexpr uint8_t FL_SOLID = 1;   // inside a particle or a static wall
constexpr uint8_t FL_SHELL = 2;   // solid with at least one fluid neighbour
constexpr int32_t OWN_FLUID = -1, OWN_WALL = -2;

// sticky device error bits
constexpr int ERR_UNSTABLE = 1, ERR_OVERFLOW = 2, ERR_FAST_PARTICLE = 4;

// ---------------------------------------------------------------- particles
struct PartState {        // per particle, FP64
    double X[3], U[3], W[3];
    double E[3];          // body axis of a spheroid (unit vector; unused for spheres)
};
struct PartStateF {       // FP32 copy read by the FP32 fluid kernels (GB300's FP64 rate is low)
    float X[3], U[3], W[3];
};
// particle record the fluid kernel of real type R reads
template <class R>
struct PartOf {
    using type = PartStateF;
};
template <>
struct PartOf<double> {
    using type = PartState;
};

// ------------------------------------------------------------ descriptors
// Everything a kernel needs to know about one box.  Lives in device memory.
struct BoxDev {
    int nx, ny, nz;
    int N;                      // nx*ny*nz (< 2^31)
    void* f;                    // populations (layout: Pop, component pairs)
    float* f0;                  // rest slot for 16-bit deviation storage, [N][2]
    void* rho[3];               // density ring: [N][2] of real each (rho^r, rho^b pairs)
    uint8_t* flags;             // [N]
    int32_t* owner;             // [N] global particle index, -1 fluid, -2 wall
    int32_t* evmark;            // [N] old owner + 3 while a remap is applied, else 0
    int pstart, np;             // global index range of this box's particles
    int has_walls;
    int vel_mode;
    int fixed;
    int implicit;               // 1: implicit particle velocity update (spheres)
    double tau[2], inv_tau[2];
    double g, rho0, scw_axis, scw_diag;
    double rho_ref[2];          // reference density of the deviation storage
    double body[3];
    double radius, mass, inertia, k_hertz, lub_cut, lub_min, nu;
    double aspect;              // spheroid semi-axes radius, radius, aspect * radius; 1 = sphere
    double rb;                  // bounding radius: max(radius, aspect * radius)
    double ipar, iperp;         // spheroid moments of inertia about / across the axis
    double c0, rho_init[2];
    double mass0[2];            // initial fluid mass
    double* mass_acc;           // [2 slots][2 components] fluid mass produced by the step kernel
    int nc[3];                  // cells per axis
    int cell_off;               // offset into the global cell arrays
    double cell_len[3];
    // remap decisions in FP32 away from the particle surface (set on the
    // host): squared reach of the scan window, sphere radius^2, the band
    // of R^2 within which the FP64 test decides, the FP32 bound beyond
    // which no node is inside a neighbour, and the spheroid form's
    // constants R^2, c^2, R^2 c^2 and band; the bounding radius in FP32
    float det_reach2, det_R2, det_band, det_qlim;
    float det_rb;
    float det_sR2, det_sc2, det_sR2c2, det_sband;
};

struct TileDev {                // one CTA work item of the fused step kernel
    int box;
    int x0, y0, z0;
    int w, h, d;
    int pad;
};

// Global per-step work lists and scratch (device memory).
struct Shared {
    PartState* part;            // [NP]
    PartStateF* partf;          // [NP] FP32 copy of part, refreshed after every MD update
    double* force;              // [NP][6] F, T accumulators
    double* force_last;         // [NP][6] coupling forces of the last step
    double* fpair;              // [NP][3] pair forces (Hertz contact, lubrication) of this step
    double* color;              // [NP]
    int* pbox;                  // [NP] box of each particle
    int* cell_count;            // [total cells]
    int* cell_start;            // [total cells + 1 per box]
    int* cell_cursor;
    int* cell_list;             // [NP]
    int* nlist;                 // [NP][NL_MAX] neighbours within 2R (claims)
    int* nlist_n;               // [NP]
    int4* events;               // [cap] (node, box, old owner, new owner)
    double* ev_rho;             // [cap][2] refill density
    int* ev_count;              // [1]
    int ev_cap;
    int4* shell_list;           // [NP][shell_cap] shell nodes of each particle (this step):
                                // (node, mask of fluid neighbours, x | y << 16, z)
    int* shell_n;               // [NP]
    int* shell_dirty;           // [NP] nonzero: rebuild the shell list (events nearby, or a new state)
    int shell_cap;
    float* xref;                // [NP][3] position at the last remap (FP32 copy)
    float* xnl;                 // [NP][3] positions at the last neighbour-list build (FP32 copy)
    int* nl_flag;               // [2] by step parity: 1 = rebuild the cell and neighbour lists in that step
    double* zdrag;              // [NP][21] drag tensor Z of the links (upper triangle, row-major; implicit update)
    double* dv;                 // [NP][6] velocity change dV of the implicit update
    int* exact;                 // [NP] 1: p owns exactly the nodes inside it at xref (remap fast path)
    int* err;                   // [1] sticky error bits
    unsigned long long* counters; // [n_boxes][2] n_cover, n_uncover
};

constexpr int NL_MAX = 32;
// The neighbour list holds every particle within the reach its users need
// (claims within 2R, the remap's scan of nodes left behind within 2R + 1.5,
// lubrication within 2R + lub_cut) plus NL_SKIN; it is rebuilt when some
// particle has moved more than NL_SKIN / 2 since the last build.
constexpr float NL_SKIN = 1.0f;
__host__ __device__ inline double nl_reach(double rb, double lub_cut) {
    return 2.0 * rb + (lub_cut > 1.55 ? lub_cut : 1.55) + (double)NL_SKIN;
}

// ------------------------------------------------------------ SplitMix64
// Steele, Lea & Flood (OOPSLA 2014): output n of a generator seeded with s
// is mix(s + (n + 1) * 0x9E3779B97F4A7C15).
__host__ __device__ inline uint64_t sm64(uint64_t s, uint64_t n) {
    uint64_t z = s + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ inline double sm64_unit(uint64_t s, uint64_t n) {
    return (double)(sm64(s, n) >> 11) * (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------------ equilibrium
// Eq. Equil with c_s^2 = 1/3:
//   zeta_i rho [1 + 3 cu + 9/2 (cu)^2 - 3/2 u^2 + 9/2 (cu)^3 - 9/2 u^2 cu].
template <class R, int I>
__device__ __forceinline__ R feq_dir(R rho, R ux, R uy, R uz, R uu) {
    R cu = R(cx(I)) * ux + R(cy(I)) * uy + R(cz(I)) * uz;
    R t = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu + R(4.5) * cu * cu * cu - R(4.5) * uu * cu;
    return wgt<R>(I) * rho * t;
}
template <class R>
__device__ __forceinline__ R feq_rt(int i, R rho, R ux, R uy, R uz) {
    R uu = ux * ux + uy * uy + uz * uz;
    R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
    R t = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu + R(4.5) * cu * cu * cu - R(4.5) * uu * cu;
    return wgt<R>(i) * rho * t;
}

// rest equilibrium as rho minus the 18 moving ones: equal to Eq. Equil in
// exact arithmetic, and sum_i f^eq_i = rho holds in finite precision too
template <class R>
__device__ __forceinline__ R feq_rest(R rho, R ux, R uy, R uz) {
    R s = R(0);
#pragma unroll
    for (int i = 1; i < 19; i++) s += feq_rt<R>(i, rho, ux, uy, uz);
    return rho - s;
}

// ----------------------------------------------------- storage policies
// Populations of component c, direction i at node n.  The two components
// of one direction and node sit side by side (a pair), so one 8-byte
// (FP32), 16-byte (FP64) or 4-byte (16-bit) access moves both:
//   FP64 / FP32: one array [19][N][2] of double / float.
//   FP16 / BF16 deviations: [18][N][2] 16-bit values d = f/zeta_i - rho_ref^c
//   for i = 1..18, and the rest population in a separate FP32 array [N][2].
// The step keeps only the 18 moving populations: the density field holds
// rho^c of every fluid node, and f_0 = rho^c - sum_{i>=1} f_i.  The rest
// slot (i = 0) only carries an imported f_0 into the density field.
// The density ring is [N][2] of the real type (FP32 for the 16-bit forms).
struct P64 {
    using real = double;
    using st = double;
    using st2 = double2;
    using real2 = double2;
    static constexpr bool dev = false;
    static constexpr int id = 0;
};
struct P32 {
    using real = float;
    using st = float;
    using st2 = float2;
    using real2 = float2;
    static constexpr bool dev = false;
    static constexpr int id = 1;
};
struct P16 {
    using real = float;
    using st = __half;
    using st2 = __half2;
    using real2 = float2;
    static constexpr bool dev = true;
    static constexpr int id = 2;
};
struct PB16 {
    using real = float;
    using st = __nv_bfloat16;
    using st2 = __nv_bfloat162;
    using real2 = float2;
    static constexpr bool dev = true;
    static constexpr int id = 3;
};

__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <class S>
__device__ __forceinline__ S from_f(float v);
template <>
__device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <class S2>
__device__ __forceinline__ S2 from_f2(float a, float b);
template <>
__device__ __forceinline__ __half2 from_f2<__half2>(float a, float b) { return __floats2half2_rn(a, b); }
template <>
__device__ __forceinline__ __nv_bfloat162 from_f2<__nv_bfloat162>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

// (red, blue) pair of the density ring or of a population slot
template <class V2, class R>
__device__ __forceinline__ V2 mk2(R a, R b) {
    V2 v;
    v.x = a;
    v.y = b;
    return v;
}

template <class P>
struct Pop {
    using R = typename P::real;
    using S = typename P::st;
    using S2 = typename P::st2;
    S* base;
    float* f0;
    size_t N;
    R ref[2];
    // deviation storage: f = zeta_i (rho_ref + d) = zeta_i d + zeta_i rho_ref,
    // one FMA per load with zr[c][w] = zeta rho_ref (w = 0 axis, 1 diagonal);
    // stores invert it with one FMA, d = f / zeta - rho_ref
    float zr[2][2];
    __device__ __forceinline__ Pop(const BoxDev& b) {
        base = reinterpret_cast<S*>(b.f);
        f0 = b.f0;
        N = (size_t)b.N;
        ref[0] = (R)b.rho_ref[0];
        ref[1] = (R)b.rho_ref[1];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            zr[c][0] = wgt<float>(1) * (float)ref[c];
            zr[c][1] = wgt<float>(7) * (float)ref[c];
        }
    }
    __device__ __forceinline__ float dev_to_f(int c, int i, S d) const {
        return fmaf(wgt<float>(i), to_f(d), zr[c][is_axis(i) ? 0 : 1]);
    }
    __device__ __forceinline__ S f_to_dev(int c, int i, float v) const {
        return from_f<S>(fmaf(v, 1.0f / wgt<float>(i), -(float)ref[c]));
    }
    // the pair (red, blue) of direction i (>= 1 for deviation storage) at node n
    __device__ __forceinline__ S2* pair(int i, size_t n) const {
        return reinterpret_cast<S2*>(base) + (size_t)(P::dev ? i - 1 : i) * N + n;
    }
    // component c of the pair of direction i at node n
    __device__ __forceinline__ S* at(int c, int i, size_t n) const {
        return base + ((size_t)(P::dev ? i - 1 : i) * N + n) * 2 + c;
    }
    __device__ __forceinline__ R load(int c, int i, int n) const {
        if constexpr (P::dev) {
            if (i == 0) return f0[(size_t)n * 2 + c];
            return dev_to_f(c, i, *at(c, i, n));
        } else {
            return *at(c, i, n);
        }
    }
    // stores v, returns the value the next load will see
    __device__ __forceinline__ R store(int c, int i, int n, R v) const {
        if constexpr (P::dev) {
            if (i == 0) {
                f0[(size_t)n * 2 + c] = v;
                return v;
            }
            const S q = f_to_dev(c, i, v);
            *at(c, i, n) = q;
            return dev_to_f(c, i, q);
        } else {
            *at(c, i, n) = v;
            return v;
        }
    }
    // load / store through a pointer to one component (direction i or
    // opp(i): opposite directions share weight and reference density)
    __device__ __forceinline__ R ld(const S* p, int c, int i) const {
        if constexpr (P::dev) return dev_to_f(c, i, *p);
        else return *p;
    }
    __device__ __forceinline__ R st(S* p, int c, int i, R v) const {
        if constexpr (P::dev) {
            const S q = f_to_dev(c, i, v);
            *p = q;
            return dev_to_f(c, i, q);
        } else {
            *p = v;
            return v;
        }
    }
    // both components through a pair pointer
    __device__ __forceinline__ void ld2(const S2* p, int i, R& a, R& b) const { cvt2(*p, i, a, b); }
    // both components of a stored pair v of direction i
    __device__ __forceinline__ void cvt2(const S2 v, int i, R& a, R& b) const {
        if constexpr (P::dev) {
            // both components in one packed FMA (the same rounding as two)
            const int k = is_axis(i) ? 0 : 1;
            const float2 r = __ffma2_rn(make_float2(wgt<float>(i), wgt<float>(i)), to_f2(v), make_float2(zr[0][k], zr[1][k]));
            a = r.x;
            b = r.y;
        } else {
            a = v.x;
            b = v.y;
        }
    }
    // stores (a, b); qa, qb: the values the next load will see
    __device__ __forceinline__ void st2(S2* p, int i, R a, R b, R& qa, R& qb) const {
        if constexpr (P::dev) {
            const int k = is_axis(i) ? 0 : 1;
            const float iw = 1.0f / wgt<float>(i);
            const float2 e = __ffma2_rn(make_float2(a, b), make_float2(iw, iw), make_float2(-(float)ref[0], -(float)ref[1]));
            const S2 q = from_f2<S2>(e.x, e.y);
            *p = q;
            const float2 r = __ffma2_rn(make_float2(wgt<float>(i), wgt<float>(i)), to_f2(q), make_float2(zr[0][k], zr[1][k]));
            qa = r.x;
            qb = r.y;
        } else {
            *p = mk2<S2>(a, b);
            qa = a;
            qb = b;
        }
    }
};

template <class P>
__host__ __device__ constexpr size_t pop_bytes(size_t N) {
    return P::dev ? (size_t)2 * 18 * N * 2 : (size_t)2 * 19 * N * sizeof(typename P::st);
}

// density ring access: the pair (rho^r, rho^b) of node n
template <class R>
struct Real2;
template <>
struct Real2<float> {
    using type = float2;
};
template <>
struct Real2<double> {
    using type = double2;
};
template <class R>
__device__ __forceinline__ typename Real2<R>::type* rpair(void* ring) {
    return reinterpret_cast<typename Real2<R>::type*>(ring);
}

// ------------------------------------------- component-pair arithmetic
// The (red, blue) values of a node in one float2 / double2.  On sm_100 and
// later one packed FP32 instruction (FADD2, FMUL2, FFMA2) does both
// components; FP64 pairs take two scalar instructions.
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 p2(double a) { return make_double2(a, a); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
// a b + c with one rounding
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
// a - b (exact product by -1, one rounding)
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 psub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ------------------------------------------------------------ helpers
__device__ __forceinline__ int wrapi(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}
// a + d for |d| <= 1 on a periodic axis of length n (no division)
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }
// Scan-window coordinates without integer division.  idx / d for
// 0 <= idx < 2^16 and 1 <= d < 2^16 is the high word of idx * m with
// m = floor((2^32 - 1) / d) + 1: m exceeds 2^32 / d by at most 1, which adds
// less than 2^-16 to idx / d, and the fraction of idx / d is at most
// 1 - 1/d < 1 - 2^-16.  When every window coordinate lies in [-n, 2n) the
// periodic wrap is a compare.  (fast: the caller has checked both;
// otherwise the division and the modulo, valid for any coordinate.)
struct WinDiv {
    int d0, d1;
    unsigned m0, m1;
    bool fast;
    __device__ __forceinline__ WinDiv(int a, int b, bool ok)
        : d0(a), d1(b), m0(0xffffffffu / (unsigned)a + 1u), m1(0xffffffffu / (unsigned)b + 1u), fast(ok) {}
    // idx = kx + d0 (ky + d1 kz)
    __device__ __forceinline__ void split(int idx, int& kx, int& ky, int& kz) const {
        const int q = fast ? (int)__umulhi((unsigned)idx, m0) : idx / d0;
        kx = idx - q * d0;
        kz = fast ? (int)__umulhi((unsigned)q, m1) : q / d1;
        ky = q - kz * d1;
    }
    __device__ __forceinline__ int wrap(int a, int n) const { return fast ? wrap1(a, n) : wrapi(a, n); }
};
// minimum image of a displacement along an axis of length L
__device__ __forceinline__ double mimg(double d, double L) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}
__device__ __forceinline__ float mimgf(float d, float L) {
    return d > 0.5f * L ? d - L : (d < -0.5f * L ? d + L : d);
}
// squared distance without contraction, so that the inside/outside test of
// a node is decided exactly as in a plain sequential evaluation
__device__ __forceinline__ double dist2_nc(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ void set_err(int* err, int bits) { atomicOr(err, bits); }

// ------------------------------------------------- particle shapes
// Spheres, or spheroids with semi-axes R, R, c = aspect R about the body
// axis e.  Inside test of a displacement d (minimum image): |d|^2 <= R^2,
// or R^2 (d.e)^2 + c^2 (|d|^2 - (d.e)^2) <= R^2 c^2, each product and sum
// rounded in this order without contraction, so that every implementation
// decides alike.
__device__ __forceinline__ bool inside_shape(const BoxDev& B, double dx, double dy, double dz, const double* e) {
    const double R2 = B.radius * B.radius;
    const double d2 = dist2_nc(dx, dy, dz);
    if (B.aspect == 1.0) return d2 <= R2;
    const double c = B.aspect * B.radius, c2 = c * c;
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, e[0]), __dmul_rn(dy, e[1])), __dmul_rn(dz, e[2]));
    const double s2 = __dmul_rn(s, s);
    return __dadd_rn(__dmul_rn(R2, s2), __dmul_rn(c2, __dsub_rn(d2, s2))) <= R2 * c2;
}
// distance from the centre to the surface along the unit vector n
__device__ __forceinline__ double support_radius(const BoxDev& B, const double* n, const double* e) {
    const double R = B.radius, c = B.aspect * B.radius;
    double t2 = n[0] * e[0] + n[1] * e[1] + n[2] * e[2];
    t2 *= t2;
    if (t2 > 1.0) t2 = 1.0;
    return 1.0 / sqrt(t2 / (c * c) + (1.0 - t2) / (R * R));
}
// contact distance of two particles along the line of centres r_hat: 2R for
// spheres, the sum of the support radii for spheroids
__device__ __forceinline__ double contact_distance(const BoxDev& B, const double* rh, const double* ep, const double* eq) {
    if (B.aspect == 1.0) return 2.0 * B.radius;
    return support_radius(B, rh, ep) + support_radius(B, rh, eq);
}

}  // namespace lbp
