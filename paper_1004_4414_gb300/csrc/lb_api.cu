// lb_api.cu -- host side of the C ABI declared in include/lbpart.h: the
// handle, the layout of the caller's device workspace, the tile plan of
// the fused step kernel, CUDA-graph capture of the time step, seeded and
// field initialisation, canonical export / import, and the observables.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lbpart.h"
#include "lb_aux.cuh"
#include "lb_ops.h"
#include "lb_structure.cuh"

using namespace lbp;

namespace {

constexpr size_t ALIGN = 256;
constexpr int SMALL_GRID = 304, SMALL_BLOCK = 256;
// line-spectrum blocks per axis of the domain-size observable
constexpr int SPEC_GRID = 1216;
// staging layout of lb_observables: phi [N], the phi sums [2 OBS_BLOCKS],
// the spectrum sums [3 SPEC_GRID], the totals [8], the coverage marks
// [np ints], then FFT scratch for lines longer than SPEC_SMEM_POINTS
constexpr size_t OBS_STAGE_FIXED = (size_t)2 * OBS_BLOCKS + 3 * SPEC_GRID + 8;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = align_up(off);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

const LbOps* ops_for(int prec) {
    switch (prec) {
        case LB_FP64: return &lb_ops_fp64;
        case LB_FP32: return &lb_ops_fp32;
        case LB_FP16_DEV: return &lb_ops_fp16;
        case LB_BF16_DEV: return &lb_ops_bf16;
        default: return nullptr;
    }
}

// spheroid aspect ratio c / R (0 in the struct means a sphere)
double aspect_of(const lb_params& p) { return p.aspect == 0.0 ? 1.0 : p.aspect; }
// bounding radius of a particle
double bound_radius(const lb_params& p) {
    const double a = aspect_of(p);
    return a > 1.0 ? a * p.radius : p.radius;
}
double particle_volume(const lb_params& p) {
    const double a = aspect_of(p);
    if (a == 1.0) return 4.0 / 3.0 * M_PI * p.radius * p.radius * p.radius;
    return 4.0 / 3.0 * M_PI * p.radius * p.radius * (a * p.radius);
}

// -1 for a count that is not a valid particle number: a volume fraction
// outside [0, 1) or NaN, or more particles than nodes
int derive_np(const lb_params& p) {
    const double N = (double)p.nx * p.ny * p.nz;
    if (p.n_particles >= 0) return p.n_particles <= N ? p.n_particles : -1;
    if (!(p.volume_fraction >= 0.0 && p.volume_fraction < 1.0)) return -1;
    const double n = std::floor(p.volume_fraction * N / particle_volume(p) + 0.5);
    return (n >= 0.0 && n <= N) ? (int)n : -1;
}

double box_color(const lb_params& p) {
    // Delta rho from the linear fit theta = 442 Delta rho + 90 (Fig. 4b)
    if (std::isfinite(p.contact_angle_deg)) return (p.contact_angle_deg - 90.0) / 442.0;
    return p.color;
}

int validate(const lb_params* bx, int nb) {
    if (!bx || nb <= 0) return LB_EINVAL;
    for (int b = 0; b < nb; b++) {
        const lb_params& p = bx[b];
        // every real parameter finite (contact_angle_deg may be NaN: use color)
        const double reals[] = {p.tau[0], p.tau[1], p.g_br, p.rho0, p.sc_weight[0], p.sc_weight[1], p.rho_init[0],
                                p.rho_init[1], p.noise_amp, p.radius, p.particle_density, p.color, p.k_hertz,
                                p.lub_cut, p.lub_min, p.mass_corr_c0, p.body_force[0], p.body_force[1],
                                p.body_force[2], p.aspect};
        for (double v : reals)
            if (!std::isfinite(v)) return LB_EINVAL;
        if (p.n_particles < 0 && !std::isfinite(p.volume_fraction)) return LB_EINVAL;
        if (p.noise_amp < 0.0 || p.k_hertz < 0.0 || p.mass_corr_c0 < 0.0) return LB_EINVAL;
        if (p.fixed_particles != 0 && p.fixed_particles != 1) return LB_EINVAL;
        if (p.nx < 1 || p.ny < 1 || p.nz < 1) return LB_EINVAL;
        if (p.nx > 65535 || p.ny > 65535 || p.nz > 65535) return LB_EINVAL;
        if ((double)p.nx * p.ny * p.nz >= 2147483647.0) return LB_EINVAL;
        if (!(p.tau[0] > 0.5) || !(p.tau[1] > 0.5)) return LB_EINVAL;
        if (!(p.rho0 > 0.0) || !(p.radius > 0.0) || !(p.particle_density > 0.0)) return LB_EINVAL;
        if (!(p.rho_init[0] > 0.0) || !(p.rho_init[1] > 0.0)) return LB_EINVAL;
        if (p.precision != bx[0].precision || !ops_for(p.precision)) return LB_EINVAL;
        if (p.vel_mode != 0 && p.vel_mode != 1) return LB_EINVAL;
        if (p.implicit_update != 0 && p.implicit_update != 1) return LB_EINVAL;
        if (p.implicit_update && aspect_of(p) != 1.0) return LB_EINVAL;  // spheres only
        if (!(p.aspect >= 0.0 && p.aspect <= 10.0) || (p.aspect != 0.0 && !(p.aspect >= 0.1))) return LB_EINVAL;
        if (derive_np(p) < 0) return LB_EINVAL;
        if (!(p.lub_min > 0.0) || !(p.lub_cut > p.lub_min)) return LB_EINVAL;
    }
    return LB_OK;
}

struct CellGeom {
    int nc[3];
    double len[3];
};
CellGeom cell_geom(const lb_params& p) {
    // cells at least as wide as the neighbour-list reach, so that the list
    // of a particle comes from the 27 cells around its own
    CellGeom g;
    const double cmin = nl_reach(bound_radius(p), p.lub_cut);
    const int L[3] = {p.nx, p.ny, p.nz};
    for (int a = 0; a < 3; a++) {
        int n = (int)std::floor(L[a] / cmin);
        if (n < 1) n = 1;
        g.nc[a] = n;
        g.len[a] = (double)L[a] / n;
    }
    return g;
}

int ev_cap_for(const lb_params& p, int np) {
    // per step a sphere moving less than one node changes at most the nodes
    // of a shell of width one around its surface
    const double R = bound_radius(p);
    const double per = 4.0 * M_PI * (R + 1.5) * (R + 1.5) * 1.5 + 64.0;
    return (int)(np * per) + 1024;
}

}  // namespace

struct lb_handle {
    int nb = 0;
    std::vector<lb_params> params;
    const LbOps* ops = nullptr;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;

    std::vector<BoxDev> hbox;
    BoxDev* d_boxes = nullptr;
    TileDev* d_tiles = nullptr;
    int max_tiles = 0, ntiles = 0, ty = 8, cz = 32;
    int split = 0;  // fused kernel with one component per thread (16-wide tiles)
    int tau1 = 0;  // every box has tau^r = tau^b = 1: the specialised fused kernel
    // the fused kernel reflects at solid neighbours itself (some box has
    // static walls, which have no link list); otherwise k_couple does it
    int reflect = 1;
    Shared sh{};
    int NP = 0, total_cells = 0;
    std::vector<int> pstart, npb, cell_off;
    std::vector<int> has_walls;
    std::vector<std::vector<double>> axes;  // per box: body axes [np][3] used by the next init
    double* stage = nullptr;
    size_t stage_doubles = 0;
    double* obs_buf = nullptr;   // [OBS_BLOCKS * OBS_W + OBS_W]
    double* mass_tmp = nullptr;  // [2]
    int64_t t = 0;
    bool initialised = false;

    cudaGraphExec_t g1[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t g6 = nullptr;
    bool graphs_ok = false;

    bool prof = false;
    std::vector<cudaEvent_t> evpool;
    int ev_used = 0;
    double prof_ms = 0.0;
    // profiling mode: an event at every phase boundary of a step, (phase,
    // event index) of each phase start; summed per phase by lb_kernel_time
    std::vector<std::pair<int, int>> phase_marks;
    double phase_ms[LB_NPHASES] = {};
    int64_t prof_fused = 0, prof_total = 0, launches_since = 0;

    int* h_err = nullptr;  // pinned mirror of the device error word
    cudaEvent_t err_ev = nullptr;
    bool err_pending = false;
    // state transfers: copies run on xstream while the conversion kernels run
    // on the handle's stream; ev_k[b] = conversion of staging half b done,
    // ev_c[b] = copy of staging half b done
    cudaStream_t xstream = nullptr;
    cudaEvent_t ev_k[2] = {nullptr, nullptr}, ev_c[2] = {nullptr, nullptr};
    // the pair forces of a step (k_md_pair) run on mdstream beside the
    // remap, shell, fused and coupling kernels: forked after the neighbour
    // list (ev_fork), joined before the velocity update (ev_join)
    cudaStream_t mdstream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<int> graph_walls;  // the per-box wall flags the graphs were captured with
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? LB_OK : LB_ECUDA; }
#define CK(x)                                          \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return LB_ECUDA;        \
    } while (0)

// Lay out the workspace (base == nullptr: only count bytes).
size_t layout(lb_handle* h, const lb_params* bx, int nb, char* base) {
    Carver cv;
    cv.base = base;
    const LbOps* ops = ops_for(bx[0].precision);
    const size_t rs = ops->real_size;
    const bool dev = bx[0].precision == LB_FP16_DEV || bx[0].precision == LB_BF16_DEV;
    int NP = 0, cells = 0, maxN = 0, maxTiles = 0, evcap = 0, maxEdge = 1;
    std::vector<BoxDev> hb(nb);
    for (int b = 0; b < nb; b++) {
        const lb_params& p = bx[b];
        const int N = p.nx * p.ny * p.nz;
        BoxDev& B = hb[b];
        memset(&B, 0, sizeof(B));
        B.nx = p.nx;
        B.ny = p.ny;
        B.nz = p.nz;
        B.N = N;
        if (dev) {
            B.f = cv.take<uint16_t>((size_t)2 * 18 * N);
            B.f0 = cv.take<float>((size_t)2 * N);
        } else {
            B.f = cv.take<char>((size_t)2 * 19 * N * rs);
        }
        for (int k = 0; k < 3; k++) B.rho[k] = cv.take<char>((size_t)2 * N * rs);
        B.flags = cv.take<uint8_t>(N);
        B.owner = cv.take<int32_t>(N);
        B.evmark = cv.take<int32_t>(N);
        B.mass_acc = cv.take<double>(4);
        const int np = derive_np(p);
        B.pstart = NP;
        B.np = np;
        NP += np;
        CellGeom cg = cell_geom(p);
        for (int a = 0; a < 3; a++) {
            B.nc[a] = cg.nc[a];
            B.cell_len[a] = cg.len[a];
        }
        B.cell_off = cells;
        cells += cg.nc[0] * cg.nc[1] * cg.nc[2];
        maxN = N > maxN ? N : maxN;
        const int e3 = p.nx > p.ny ? (p.nx > p.nz ? p.nx : p.nz) : (p.ny > p.nz ? p.ny : p.nz);
        maxEdge = e3 > maxEdge ? e3 : maxEdge;
        // the most tiles any block shape makes: 32 x 4 or (split) 16 x 8 nodes, one plane each
        const int t32 = ((p.nx + 31) / 32) * ((p.ny + 3) / 4), t16 = ((p.nx + 15) / 16) * ((p.ny + 7) / 8);
        maxTiles += (t32 > t16 ? t32 : t16) * p.nz;
        evcap += ev_cap_for(p, np);
    }
    Shared sh{};
    const int NPa = NP > 0 ? NP : 1;
    sh.part = cv.take<PartState>(NPa);
    sh.partf = cv.take<PartStateF>(NPa);
    sh.force = cv.take<double>((size_t)NPa * 6);
    sh.force_last = cv.take<double>((size_t)NPa * 6);
    sh.fpair = cv.take<double>((size_t)NPa * 3);
    sh.color = cv.take<double>(NPa);
    sh.pbox = cv.take<int>(NPa);
    sh.cell_count = cv.take<int>(cells);
    sh.cell_start = cv.take<int>(cells);
    sh.cell_cursor = cv.take<int>(cells);
    sh.cell_list = cv.take<int>(NPa);
    sh.nlist = cv.take<int>((size_t)NPa * NL_MAX);
    sh.nlist_n = cv.take<int>(NPa);
    sh.events = cv.take<int4>(evcap);
    sh.ev_rho = cv.take<double>((size_t)evcap * 2);
    sh.ev_count = cv.take<int>(1);
    sh.ev_cap = evcap;
    {
        // shell nodes of one sphere: a one-node layer around its surface
        double rmax = 0.0;
        for (int b = 0; b < nb; b++) rmax = bound_radius(bx[b]) > rmax ? bound_radius(bx[b]) : rmax;
        sh.shell_cap = (int)(12.0 * (rmax + 1.0) * (rmax + 1.0)) + 64;
    }
    sh.shell_list = cv.take<int4>((size_t)NPa * sh.shell_cap);
    sh.shell_n = cv.take<int>(NPa);
    sh.shell_dirty = cv.take<int>(NPa);
    sh.xref = cv.take<float>((size_t)NPa * 3);
    sh.exact = cv.take<int>(NPa);
    sh.xnl = cv.take<float>((size_t)NPa * 3);
    sh.nl_flag = cv.take<int>(2);
    sh.zdrag = cv.take<double>((size_t)NPa * 21);
    sh.dv = cv.take<double>((size_t)NPa * 6);
    sh.err = cv.take<int>(1);
    sh.counters = cv.take<unsigned long long>((size_t)nb * 2);
    BoxDev* d_boxes = cv.take<BoxDev>(nb);
    TileDev* d_tiles = cv.take<TileDev>(maxTiles);
    // import/export and init need 5 N + 9 np; lb_observables N + fixed sums +
    // np / 2 for the marks + FFT scratch of at least one line beyond
    // SPEC_SMEM_POINTS (3 n complex values)
    const size_t stage_doubles = (size_t)5 * maxN + (size_t)9 * NPa + OBS_STAGE_FIXED + (size_t)6 * maxEdge + 64;
    double* stage = cv.take<double>(stage_doubles);
    double* obs = cv.take<double>((size_t)OBS_BLOCKS * OBS_W + OBS_W);
    double* mtmp = cv.take<double>(2);
    if (h && base) {
        h->hbox = hb;
        h->sh = sh;
        h->d_boxes = d_boxes;
        h->d_tiles = d_tiles;
        h->max_tiles = maxTiles;
        h->NP = NP;
        h->total_cells = cells;
        h->stage = stage;
        h->stage_doubles = stage_doubles;
        h->obs_buf = obs;
        h->mass_tmp = mtmp;
    }
    return align_up(cv.off);
}

void fill_params(lb_handle* h) {
    for (int b = 0; b < h->nb; b++) {
        const lb_params& p = h->params[b];
        BoxDev& B = h->hbox[b];
        B.has_walls = h->has_walls[b];
        B.vel_mode = p.vel_mode;
        B.fixed = p.fixed_particles;
        B.implicit = p.implicit_update;
        for (int c = 0; c < 2; c++) {
            B.tau[c] = p.tau[c];
            B.inv_tau[c] = 1.0 / p.tau[c];
            B.rho_ref[c] = p.rho_init[c];
            B.rho_init[c] = p.rho_init[c];
        }
        B.g = p.g_br;
        B.rho0 = p.rho0;
        B.scw_axis = p.sc_weight[0];
        B.scw_diag = p.sc_weight[1];
        for (int a = 0; a < 3; a++) B.body[a] = p.body_force[a];
        B.radius = p.radius;
        B.aspect = aspect_of(p);
        B.rb = bound_radius(p);
        B.mass = p.particle_density * particle_volume(p);
        B.inertia = 0.4 * B.mass * p.radius * p.radius;
        // spheroid (semi-axes R, R, c): about the axis 2/5 m R^2, across it
        // 1/5 m (R^2 + c^2)
        B.ipar = B.inertia;
        B.iperp = 0.2 * B.mass * (p.radius * p.radius + (B.aspect * p.radius) * (B.aspect * p.radius));
        B.k_hertz = p.k_hertz;
        B.lub_cut = p.lub_cut;
        B.lub_min = p.lub_min;
        B.nu = (1.0 / 3.0) * (0.5 * (p.tau[0] + p.tau[1]) - 0.5);
        B.c0 = p.mass_corr_c0;
        {
            // FP32 positions near L are off by up to about L * 2^-24 per
            // axis (eps_pos / 2).  A squared distance d^2 <= (R + 1.5)^2
            // from them is off by at most 2 |d| sqrt(3) eps_pos / 2 (under
            // 11.3 eps_pos) plus the FP32 rounding of the window offsets and
            // of the sum (under 1e-5 R^2).  The band keeps every FP32 remap
            // decision more than twice that away from the surface (the FP64
            // test decides within it); the neighbour bound qlim, whose
            // distances carry the error of both centres, takes two bands.
            const double R = B.rb, R2 = B.radius * B.radius;
            const int nmax = p.nx > p.ny ? (p.nx > p.nz ? p.nx : p.nz) : (p.ny > p.nz ? p.ny : p.nz);
            const double eps_pos = 1.2e-7 * (double)nmax;
            B.det_reach2 = (float)((R + 1.5) * (R + 1.5));
            B.det_rb = (float)R;
            B.det_R2 = (float)R2;
            B.det_band = (float)(1e-4 + 2e-5 * R * R + 4.0 * (R + 1.5) * eps_pos);
            B.det_qlim = (float)(R * R) + 2.0f * B.det_band;
            // spheroid form F = R^2 (d.e)^2 + c^2 (|d|^2 - (d.e)^2) against
            // R^2 c^2: |grad F| <= gmax = 2 max(R^2, c^2) |d| within the
            // window, so the position error (sqrt(3) eps_pos / 2) moves F by
            // under 0.87 gmax eps_pos; the FP32 axis and the rounding of F's
            // terms (each below max(R^2, c^2) |d|^2 near the surface) add
            // under 1e-3 + 1e-6 R^2 c^2.  The band is twice that.
            const double cRd = B.aspect * B.radius;
            const double gmax = 2.0 * (R2 > cRd * cRd ? R2 : cRd * cRd) * (R + 1.5);
            const float cR = (float)cRd;
            B.det_sR2 = (float)R2;
            B.det_sc2 = cR * cR;
            B.det_sR2c2 = B.det_sR2 * B.det_sc2;
            B.det_sband = (float)(2e-3 + 2.0 * gmax * eps_pos + 2e-6 * R2 * cRd * cRd);
        }
    }
}

int upload_boxes(lb_handle* h) {
    CK(cudaMemcpyAsync(h->d_boxes, h->hbox.data(), sizeof(BoxDev) * h->nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int build_tiles(lb_handle* h) {
    std::vector<TileDev> tl;
    const int tw = h->split ? 16 : 32;  // tile width in x
    for (int b = 0; b < h->nb; b++) {
        const BoxDev& B = h->hbox[b];
        for (int z0 = 0; z0 < B.nz; z0 += h->cz)
            for (int y0 = 0; y0 < B.ny; y0 += h->ty)
                for (int x0 = 0; x0 < B.nx; x0 += tw) {
                    TileDev t;
                    t.box = b;
                    t.x0 = x0;
                    t.y0 = y0;
                    t.z0 = z0;
                    t.w = B.nx - x0 < tw ? B.nx - x0 : tw;
                    t.h = B.ny - y0 < h->ty ? B.ny - y0 : h->ty;
                    t.d = B.nz - z0 < h->cz ? B.nz - z0 : h->cz;
                    t.pad = 0;
                    tl.push_back(t);
                }
    }
    if ((int)tl.size() > h->max_tiles) return LB_ENOMEM;
    h->ntiles = (int)tl.size();
    CK(cudaMemcpyAsync(h->d_tiles, tl.data(), sizeof(TileDev) * tl.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

// all kernels of one time step t
// profiling: an event on the stream (from the handle's pool)
int prof_event(lb_handle* h, int* idx) {
    if (h->ev_used + 1 > (int)h->evpool.size()) {
        for (int k = 0; k < 64; k++) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            h->evpool.push_back(e);
        }
    }
    *idx = h->ev_used++;
    CK(cudaEventRecord(h->evpool[*idx], h->stream));
    return LB_OK;
}

int enqueue_step(lb_handle* h, int64_t t, bool prof) {
    cudaStream_t st = h->stream;
    // phase boundaries (profiling only): phase k runs between marks k and k + 1
    int evi = 0;
    auto mark = [&](int phase) -> int {
        if (!prof) return LB_OK;
        int rc = prof_event(h, &evi);
        if (rc == LB_OK) h->phase_marks.push_back({phase, evi});
        return rc;
    };
    if (mark(0) != LB_OK) return LB_ECUDA;
    const int par = (int)(t & 1), rc = (int)(t % 3), rn = (int)((t + 1) % 3), rz = (int)((t + 2) % 3);
    const int mcur = (int)(t & 1), mnext = (int)((t + 1) & 1);
    const int NP = h->NP;
    int launches = 0;
    h->reflect = 0;
    for (int b = 0; b < h->nb; b++)
        if (h->has_walls[b]) h->reflect = 1;
    k_step_begin<<<SMALL_GRID, SMALL_BLOCK, 0, st>>>(h->d_boxes, h->nb, h->sh, h->total_cells, mnext, par);
    launches++;
    if (NP > 0) {
        const int pg = (NP + 255) / 256;
        k_cell_count<<<pg, 256, 0, st>>>(h->d_boxes, h->sh, NP, par);
        k_cell_scan<<<h->nb, 1024, 0, st>>>(h->d_boxes, h->sh, par);
        k_cell_fill<<<pg, 256, 0, st>>>(h->d_boxes, h->sh, NP, par);
        k_nlist<<<(NP + NLIST_WARPS - 1) / NLIST_WARPS, 32 * NLIST_WARPS, 0, st>>>(h->d_boxes, h->sh, NP, par);
        // the pair forces read only the positions, velocities and
        // neighbour lists, which nothing changes before the velocity update
        CK(cudaEventRecord(h->ev_fork, st));
        CK(cudaStreamWaitEvent(h->mdstream, h->ev_fork, 0));
        k_md_pair<<<(NP + MD_WARPS - 1) / MD_WARPS, 32 * MD_WARPS, 0, h->mdstream>>>(h->d_boxes, h->sh, NP);
        CK(cudaEventRecord(h->ev_join, h->mdstream));
        if (mark(1) != LB_OK) return LB_ECUDA;
        k_remap_detect<<<NP, 32 * DETECT_WARPS, 0, st>>>(h->d_boxes, h->sh, NP);
        if (mark(2) != LB_OK) return LB_ECUDA;
        k_remap_mark<<<SMALL_GRID, SMALL_BLOCK, 0, st>>>(h->d_boxes, h->sh);
        CK(cudaGetLastError());
        CK(h->ops->remap_apply(par, st, h->d_boxes, h->sh, rc, mcur));
        CK(h->ops->remap_finish(st, h->d_boxes, h->sh, rc));
        if (mark(3) != LB_OK) return LB_ECUDA;
        CK(h->ops->shell_density(st, h->d_boxes, h->sh, rc, NP));
        launches += 10;
    }
    for (int b = 0; b < h->nb; b++)
        if (h->has_walls[b]) {
            CK(h->ops->wall_shell(st, h->d_boxes, b, rc));
            launches++;
        }
    if (mark(4) != LB_OK) return LB_ECUDA;
    CK(h->ops->step(par, h->ty, h->split, h->tau1, h->reflect, h->ntiles, st, h->d_boxes, h->d_tiles, h->sh, rc, rn, rz, mnext));
    launches++;
    if (prof) h->prof_fused++;
    if (mark(5) != LB_OK) return LB_ECUDA;
    if (NP > 0) {
        const int pg = (NP + 255) / 256;
        int impl = 0;
        for (const auto& p : h->params) impl |= p.implicit_update;
        CK(h->ops->couple(st, h->d_boxes, h->sh, rc, rn, mnext, par, h->reflect, impl, NP));
        if (mark(6) != LB_OK) return LB_ECUDA;
        CK(cudaStreamWaitEvent(st, h->ev_join, 0));
        if (impl) {
            // implicit update: velocities, the fluid's share on the links, positions
            k_md_solve<<<pg, 256, 0, st>>>(h->d_boxes, h->sh, NP);
            CK(h->ops->couple_correct(st, h->d_boxes, h->sh, rc, rn, mnext, par, h->reflect, NP));
            k_md_move<<<pg, 256, 0, st>>>(h->d_boxes, h->sh, NP, par);
            launches += 4;
        } else {
            k_md_integrate<<<pg, 256, 0, st>>>(h->d_boxes, h->sh, NP, par);
            launches += 2;
        }
    }
    if (mark(LB_NPHASES) != LB_OK) return LB_ECUDA;  // end of the step
    h->launches_since = launches;
    if (prof) h->prof_total += launches;
    CK(cudaGetLastError());
    return LB_OK;
}

void destroy_graphs(lb_handle* h) {
    for (auto& g : h->g1)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (h->g6) {
        cudaGraphExecDestroy(h->g6);
        h->g6 = nullptr;
    }
    h->graphs_ok = false;
}

int capture(lb_handle* h, int64_t t0, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LB_OK;
    for (int k = 0; k < nsteps && rc == LB_OK; k++) rc = enqueue_step(h, t0 + k, false);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != LB_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return LB_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return cuda_rc(e);
}

int build_graphs(lb_handle* h) {
    destroy_graphs(h);
    for (int k = 0; k < 6; k++) {
        int rc = capture(h, k, 1, &h->g1[k]);
        if (rc != LB_OK) return rc;
    }
    int rc = capture(h, 0, 6, &h->g6);
    if (rc != LB_OK) return rc;
    h->graphs_ok = true;
    h->graph_walls = h->has_walls;
    return LB_OK;
}

int map_err(int bits) {
    if (bits & ERR_OVERFLOW) return LB_EOVERFLOW;
    if (bits & (ERR_UNSTABLE | ERR_FAST_PARTICLE)) return LB_EUNSTABLE;
    return LB_OK;
}

int read_err(lb_handle* h) {
    int v = 0;
    CK(cudaMemcpyAsync(&v, h->sh.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return map_err(v);
}

// Random sequential addition of the spheres of one box (host; stream 0 of
// the box seed): candidate centre = L * u for three successive draws,
// accepted when every earlier centre is at least 2R away (minimum image).
// A cell grid only speeds up the search; decisions are those of the plain
// all-pairs test.
int rsa_place(const lb_params& p, int np, uint64_t s0, std::vector<double>& parts) {
    parts.assign((size_t)np * 9, 0.0);
    const double L[3] = {(double)p.nx, (double)p.ny, (double)p.nz};
    const double rb = bound_radius(p);
    const double dmin2 = 4.0 * rb * rb;
    int gc[3];
    for (int a = 0; a < 3; a++) {
        gc[a] = (int)std::floor(L[a] / (2.0 * rb));
        if (gc[a] < 1) gc[a] = 1;
    }
    std::vector<std::vector<int>> grid((size_t)gc[0] * gc[1] * gc[2]);
    auto cell = [&](const double* c, int a) {
        int v = (int)(c[a] / L[a] * gc[a]);
        return v < 0 ? 0 : (v >= gc[a] ? gc[a] - 1 : v);
    };
    auto mi = [](double d, double Lx) { return d > 0.5 * Lx ? d - Lx : (d < -0.5 * Lx ? d + Lx : d); };
    uint64_t draw = 0;
    int placed = 0;
    for (int64_t attempt = 0; placed < np; attempt++) {
        if (attempt >= 1000000) return LB_EPLACE;
        double c[3];
        for (int a = 0; a < 3; a++) c[a] = L[a] * sm64_unit(s0, draw++);
        bool ok = true;
        int ci[3];
        for (int a = 0; a < 3; a++) ci[a] = cell(c, a);
        const int rng[3] = {gc[0] >= 3 ? 1 : gc[0], gc[1] >= 3 ? 1 : gc[1], gc[2] >= 3 ? 1 : gc[2]};
        for (int dz = (gc[2] >= 3 ? -1 : 0); dz <= (gc[2] >= 3 ? 1 : gc[2] - 1) && ok; dz++)
            for (int dy = (gc[1] >= 3 ? -1 : 0); dy <= (gc[1] >= 3 ? 1 : gc[1] - 1) && ok; dy++)
                for (int dx = (gc[0] >= 3 ? -1 : 0); dx <= (gc[0] >= 3 ? 1 : gc[0] - 1) && ok; dx++) {
                    const int cx_ = gc[0] >= 3 ? (ci[0] + dx + gc[0]) % gc[0] : dx;
                    const int cy_ = gc[1] >= 3 ? (ci[1] + dy + gc[1]) % gc[1] : dy;
                    const int cz_ = gc[2] >= 3 ? (ci[2] + dz + gc[2]) % gc[2] : dz;
                    for (int q : grid[(size_t)cx_ + gc[0] * ((size_t)cy_ + gc[1] * cz_)]) {
                        const double ddx = mi(c[0] - parts[9 * q + 0], L[0]);
                        const double ddy = mi(c[1] - parts[9 * q + 1], L[1]);
                        const double ddz = mi(c[2] - parts[9 * q + 2], L[2]);
                        const double a2 = ddx * ddx, b2 = ddy * ddy, c2 = ddz * ddz;
                        if ((a2 + b2) + c2 < dmin2) {
                            ok = false;
                            break;
                        }
                    }
                }
        (void)rng;
        if (!ok) continue;
        for (int a = 0; a < 3; a++) parts[9 * placed + a] = c[a];
        grid[(size_t)cell(c, 0) + gc[0] * ((size_t)cell(c, 1) + gc[1] * cell(c, 2))].push_back(placed);
        placed++;
    }
    return LB_OK;
}

// status, populations and density of box b at t = 0
int init_box(lb_handle* h, int b, const double* parts_host, const int32_t* walls_host, const double* rho_dev,
             const double* u_dev, uint64_t s_red, uint64_t s_blue, double noise) {
    cudaStream_t st = h->stream;
    BoxDev& B = h->hbox[b];
    const int N = B.N, np = B.np;
    // particles
    if (np > 0) {
        std::vector<PartState> ps(np);
        std::vector<int> pb(np, b);
        std::vector<double> col(np, box_color(h->params[b]));
        const std::vector<double>& ax = h->axes[b];
        for (int q = 0; q < np; q++)
            for (int a = 0; a < 3; a++) {
                ps[q].X[a] = parts_host[9 * q + a];
                ps[q].U[a] = parts_host[9 * q + 3 + a];
                ps[q].W[a] = parts_host[9 * q + 6 + a];
                ps[q].E[a] = ax[3 * q + a];
            }
        CK(cudaMemcpyAsync(h->sh.part + B.pstart, ps.data(), sizeof(PartState) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(h->sh.pbox + B.pstart, pb.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(h->sh.color + B.pstart, col.data(), sizeof(double) * np, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(h->sh.force + (size_t)B.pstart * 6, 0, sizeof(double) * 6 * np, st));
        CK(cudaMemsetAsync(h->sh.force_last + (size_t)B.pstart * 6, 0, sizeof(double) * 6 * np, st));
        k_part_to_float<<<(np + 255) / 256, 256, 0, st>>>(h->sh, B.pstart, np);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
    }
    // walls (owner -2) or fluid
    h->has_walls[b] = 0;
    if (walls_host) {
        std::vector<int32_t> own(N);
        for (int n = 0; n < N; n++) {
            own[n] = walls_host[n] == OWN_WALL ? OWN_WALL : OWN_FLUID;
            if (own[n] == OWN_WALL) h->has_walls[b] = 1;
        }
        CK(cudaMemcpyAsync(B.owner, own.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    } else {
        k_fill<int32_t><<<SMALL_GRID * 4, 256, 0, st>>>(B.owner, OWN_FLUID, (size_t)N);
    }
    // claims: smallest distance, then lowest index (scratch in the stage;
    // rho_dev / u_dev must not overlap it: they are placed after it)
    unsigned long long* key = reinterpret_cast<unsigned long long*>(h->stage);
    int* idb = reinterpret_cast<int*>(h->stage + N);
    k_fill<unsigned long long><<<SMALL_GRID * 4, 256, 0, st>>>(key, 0x7FF0000000000000ull, (size_t)N);
    k_fill<int><<<SMALL_GRID * 4, 256, 0, st>>>(idb, 0x7fffffff, (size_t)N);
    h->hbox[b].has_walls = h->has_walls[b];
    fill_params(h);
    int rc = upload_boxes(h);
    if (rc != LB_OK) return rc;
    if (np > 0) {
        const int g = (np + 3) / 4;
        k_claim<1><<<g, 128, 0, st>>>(h->d_boxes, h->sh, b, key, idb);
        k_claim<2><<<g, 128, 0, st>>>(h->d_boxes, h->sh, b, key, idb);
    }
    k_owner_from_claims<<<SMALL_GRID * 4, 256, 0, st>>>(h->d_boxes, b, idb);
    k_shell_all<<<SMALL_GRID * 4, 256, 0, st>>>(h->d_boxes, b);
    CK(cudaGetLastError());
    // density ring, marks
    for (int k = 0; k < 3; k++) CK(cudaMemsetAsync(B.rho[k], 0, (size_t)2 * N * h->ops->real_size, st));
    CK(cudaMemsetAsync(B.evmark, 0, sizeof(int32_t) * N, st));
    CK(cudaMemsetAsync(h->mass_tmp, 0, 2 * sizeof(double), st));
    CK(h->ops->init_pop(st, h->d_boxes, b, rho_dev, u_dev, s_red, s_blue, noise, 0, h->mass_tmp));
    double m[2];
    CK(cudaMemcpyAsync(m, h->mass_tmp, sizeof(m), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    B.mass0[0] = m[0];
    B.mass0[1] = m[1];
    double ma[4] = {m[0], m[1], 0.0, 0.0};
    CK(cudaMemcpyAsync(B.mass_acc, ma, sizeof(ma), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->sh.counters + 2 * b, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(h->sh.err, 0, sizeof(int), st));
    rc = upload_boxes(h);
    if (rc != LB_OK) return rc;
    return LB_OK;
}

int after_init(lb_handle* h, int64_t t) {
    h->t = t;
    h->initialised = true;
    h->err_pending = false;
    // every shell list is rebuilt at the first step of a new state
    if (h->NP > 0) {
        CK(cudaMemsetAsync(h->sh.shell_dirty, 1, sizeof(int) * h->NP, h->stream));
        // and the first remap scans every particle's whole window, and the
        // first step builds the cell and neighbour lists
        CK(cudaMemsetAsync(h->sh.exact, 0, sizeof(int) * h->NP, h->stream));
        CK(cudaMemsetAsync(h->sh.nl_flag, 1, 2 * sizeof(int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    // graphs bake in the per-box wall flags (the wall-shell launches and the
    // reflection mode), so they are rebuilt only when those changed; the
    // legacy default stream cannot be captured, steps then launch directly
    if (h->stream == nullptr) {
        destroy_graphs(h);
        return LB_OK;
    }
    if (h->graphs_ok && h->graph_walls == h->has_walls) return LB_OK;
    return build_graphs(h);
}

// Domain size (Eq. eq:domsize) and interface coverage of box b on the
// device (lb_structure.cuh); phi_out (host, N doubles) receives phi if not
// NULL.  Synchronises the stream.
int structure_obs(lb_handle* h, int box, double L[3], double* coverage, double* phi_out) {
    const BoxDev& B = h->hbox[box];
    cudaStream_t st = h->stream;
    const size_t N = (size_t)B.N;
    const int rc = (int)(h->t % 3);
    double* phi = h->stage;
    double* phisum = phi + N;
    double* specsum = phisum + 2 * OBS_BLOCKS;
    double* tot = specsum + 3 * SPEC_GRID;
    int* marks = reinterpret_cast<int*>(tot + 8);
    double2* scratch = reinterpret_cast<double2*>(tot + 8 + ((size_t)B.np + 1) / 2 + 2);
    scratch = reinterpret_cast<double2*>(((uintptr_t)scratch + 15) & ~(uintptr_t)15);
    const size_t scratch_c2 = (h->stage_doubles - (size_t)((double*)scratch - h->stage)) / 2;  // double2 slots
    CK(h->ops->phi_field(st, h->d_boxes, box, rc, phi, phisum));
    k_sum_columns<<<1, 32, 0, st>>>(phisum, OBS_BLOCKS, 2, 2, tot);
    const int dims[3] = {B.nx, B.ny, B.nz};
    int grid[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) {
        const int n = dims[a];
        const Radices rad = radices_of(n);
        const int nlines = (int)(N / (size_t)n);
        if (n <= SPEC_SMEM_POINTS) {
            int W = SPEC_SMEM_POINTS / n;
            if (W > nlines) W = nlines;
            const int ngroups = (nlines + W - 1) / W;
            const int G = ngroups < SPEC_GRID ? ngroups : SPEC_GRID;
            const size_t smem = (2 * (size_t)W * n + n) * sizeof(double2);
            k_line_spectrum<true><<<G, SPEC_THREADS, smem, st>>>(phi, B.nx, B.ny, B.nz, a, W, rad, nullptr,
                                                                  specsum + a * SPEC_GRID);
            grid[a] = G;
        } else {
            const size_t per = 3 * (size_t)n;  // double2 per block
            size_t G = scratch_c2 / per;
            if (G > (size_t)SPEC_GRID) G = SPEC_GRID;
            if (G > (size_t)nlines) G = nlines;
            if (G < 1) return LB_ENOMEM;
            k_line_spectrum<false><<<(int)G, SPEC_THREADS, 0, st>>>(phi, B.nx, B.ny, B.nz, a, 1, rad, scratch,
                                                                     specsum + a * SPEC_GRID);
            grid[a] = (int)G;
        }
        CK(cudaGetLastError());
        k_sum_columns<<<1, 32, 0, st>>>(specsum + a * SPEC_GRID, grid[a], 1, 1, tot + 2 + a);
    }
    if (B.np > 0) {
        CK(cudaMemsetAsync(marks, 0, sizeof(int) * B.np, st));
        CK(h->ops->coverage_marks(st, h->d_boxes, box, rc, marks));
        k_count_both<<<1, 256, 0, st>>>(marks, B.np, tot + 5);
    }
    CK(cudaGetLastError());
    double v[6] = {0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(v, tot, sizeof(double) * (B.np > 0 ? 6 : 5), cudaMemcpyDeviceToHost, st));
    if (phi_out) CK(cudaMemcpyAsync(phi_out, phi, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // sum phi'^2 = sum phi^2 - N <phi>^2; <k_a^2> = spectrum_a / (n_a sum phi'^2)
    const double mean = v[0] / (double)N;
    const double var = v[1] - (double)N * mean * mean;
    for (int a = 0; a < 3; a++) {
        const double k2 = v[2 + a] / ((double)dims[a] * var);
        L[a] = (var > 0.0 && k2 > 0.0) ? 2.0 * M_PI / std::sqrt(k2) : NAN;
    }
    *coverage = B.np > 0 ? v[5] / (double)B.np : 0.0;
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_strerror(int code) {
    switch (code) {
        case LB_OK: return "ok";
        case LB_EINVAL: return "invalid argument";
        case LB_ENOMEM: return "workspace too small";
        case LB_ECUDA: return "CUDA runtime error";
        case LB_EUNSTABLE: return "unstable: non-finite density, |u| >= 0.5, or a particle faster than 1 node/step";
        case LB_EPLACE: return "random sequential addition could not place the spheres";
        case LB_ETIMEOUT: return "bounded device wait gave up";
        case LB_EOVERFLOW: return "a fixed-capacity device list overflowed";
        default: return "unknown error";
    }
}

int lb_workspace_bytes(const lb_params* boxes, int32_t n_boxes, size_t* bytes) {
    if (!bytes) return LB_EINVAL;
    int rc = validate(boxes, n_boxes);
    if (rc != LB_OK) return rc;
    *bytes = layout(nullptr, boxes, n_boxes, nullptr);
    return LB_OK;
}

int lb_create(const lb_params* boxes, int32_t n_boxes, void* d_workspace, size_t bytes, void* cuda_stream,
              lb_handle** out) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    int rc = validate(boxes, n_boxes);
    if (rc != LB_OK) return rc;
    if (!d_workspace || ((uintptr_t)d_workspace % ALIGN) != 0) return LB_EINVAL;
    const size_t need = layout(nullptr, boxes, n_boxes, nullptr);
    if (bytes < need) return LB_ENOMEM;
    lb_handle* h = new lb_handle();
    h->nb = n_boxes;
    h->params.assign(boxes, boxes + n_boxes);
    h->ops = ops_for(boxes[0].precision);
    h->stream = (cudaStream_t)cuda_stream;
    h->ws = (char*)d_workspace;
    h->ws_bytes = bytes;
    h->has_walls.assign(n_boxes, 0);
    h->tau1 = 1;
    for (int b = 0; b < n_boxes; b++)
        if (boxes[b].tau[0] != 1.0 || boxes[b].tau[1] != 1.0) h->tau1 = 0;
    layout(h, boxes, n_boxes, h->ws);
    fill_params(h);
    h->axes.resize(n_boxes);
    for (int b = 0; b < n_boxes; b++) {
        h->axes[b].assign((size_t)3 * h->hbox[b].np, 0.0);
        for (int q = 0; q < h->hbox[b].np; q++) h->axes[b][3 * q + 2] = 1.0;
    }
    if (h->ops->setup() != cudaSuccess ||
        cudaFuncSetAttribute(k_line_spectrum<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(3 * SPEC_SMEM_POINTS * sizeof(double2))) != cudaSuccess ||
        cudaHostAlloc((void**)&h->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->err_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->xstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_k[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_k[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_c[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_c[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->mdstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        lb_destroy(h);
        return LB_ECUDA;
    }
    *h->h_err = 0;
    // default tiling: 8 rows per CTA; z chunks so that there are >= 4 waves of CTAs on 152 SMs
    h->ty = 8;
    long long cols = 0;
    int maxnz = 1;
    for (auto& p : h->params) {
        cols += (long long)((p.nx + 31) / 32) * ((p.ny + 7) / 8);
        maxnz = p.nz > maxnz ? p.nz : maxnz;
    }
    int cz = maxnz;
    while (cz > 8 && cols * ((maxnz + cz - 1) / cz) < 152 * 8) cz = (cz + 1) / 2;
    h->cz = cz;
    rc = upload_boxes(h);
    if (rc == LB_OK) rc = build_tiles(h);
    if (rc == LB_OK) {
        CK(cudaMemsetAsync(h->sh.err, 0, sizeof(int), h->stream));
        CK(cudaMemsetAsync(h->sh.counters, 0, sizeof(unsigned long long) * 2 * h->nb, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (rc != LB_OK) {
        lb_destroy(h);
        return rc;
    }
    *out = h;
    return LB_OK;
}

int lb_init_from_seed(lb_handle* h, uint64_t seed) {
    if (!h) return LB_EINVAL;
    for (int b = 0; b < h->nb; b++) {
        const uint64_t sb = seed + (uint64_t)b;
        const uint64_t s0 = sm64(sb, 0), s_red = sm64(sb, 1), s_blue = sm64(sb, 2);
        std::vector<double> parts;
        int rc = rsa_place(h->params[b], h->hbox[b].np, s0, parts);
        if (rc != LB_OK) return rc;
        // spheroid axes from stream 3: z = 2u - 1, phi = 2 pi u' (draws
        // 2q, 2q + 1), e = (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z)
        if (aspect_of(h->params[b]) != 1.0) {
            const uint64_t se = sm64(sb, 3);
            std::vector<double>& ax = h->axes[b];
            for (int q = 0; q < h->hbox[b].np; q++) {
                const double zc = 2.0 * sm64_unit(se, 2 * (uint64_t)q) - 1.0;
                const double ph = 2.0 * M_PI * sm64_unit(se, 2 * (uint64_t)q + 1);
                const double rr = std::sqrt(1.0 - zc * zc);
                ax[3 * q + 0] = rr * std::cos(ph);
                ax[3 * q + 1] = rr * std::sin(ph);
                ax[3 * q + 2] = zc;
            }
        }
        rc = init_box(h, b, parts.data(), nullptr, nullptr, nullptr, s_red, s_blue, h->params[b].noise_amp);
        if (rc != LB_OK) return rc;
    }
    return after_init(h, 0);
}

int lb_init_fields(lb_handle* h, int32_t box, const double* rho, const double* u, const double* particles,
                   const int32_t* walls) {
    if (!h || box < 0 || box >= h->nb || !rho) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    if (B.np > 0 && !particles) return LB_EINVAL;
    const size_t N = (size_t)B.N;
    // The node status is built first (its claim scratch occupies the first
    // 1.5 N doubles of the stage) with uniform rho_init populations; then
    // the fields are copied into the stage (rho at [0, 2N), u at [2N, 5N))
    // and the populations are rebuilt from them.
    double* rho_dev = h->stage;
    double* u_dev = u ? h->stage + 2 * N : nullptr;
    int rc;
    {
        cudaStream_t st = h->stream;
        rc = init_box(h, box, particles, walls, nullptr, nullptr, 0, 0, 0.0);
        if (rc != LB_OK) return rc;
        CK(cudaMemcpyAsync(rho_dev, rho, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, st));
        if (u) CK(cudaMemcpyAsync(u_dev, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(h->mass_tmp, 0, 2 * sizeof(double), st));
        CK(h->ops->init_pop(st, h->d_boxes, box, rho_dev, u_dev, 0, 0, 0.0, 0, h->mass_tmp));
        double m[2];
        CK(cudaMemcpyAsync(m, h->mass_tmp, sizeof(m), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        BoxDev& Bw = h->hbox[box];
        Bw.mass0[0] = m[0];
        Bw.mass0[1] = m[1];
        double ma[4] = {m[0], m[1], 0.0, 0.0};
        CK(cudaMemcpyAsync(Bw.mass_acc, ma, sizeof(ma), cudaMemcpyHostToDevice, st));
        rc = upload_boxes(h);
        if (rc != LB_OK) return rc;
    }
    return after_init(h, 0);
}

int lb_step(lb_handle* h, int64_t n) {
    if (!h || n < 0) return LB_EINVAL;
    if (!h->initialised) return LB_EINVAL;
    // report a device error seen by an earlier call that has finished
    if (h->err_pending && cudaEventQuery(h->err_ev) == cudaSuccess) {
        h->err_pending = false;
        int e = map_err(*h->h_err);
        if (e != LB_OK) return e;
    }
    if (n == 0) return LB_OK;
    while (n > 0) {
        if (h->prof || !h->graphs_ok) {
            int rc = enqueue_step(h, h->t, h->prof);
            if (rc != LB_OK) return rc;
            h->t++;
            n--;
        } else if (h->t % 6 == 0 && n >= 6) {
            CK(cudaGraphLaunch(h->g6, h->stream));
            h->t += 6;
            n -= 6;
        } else {
            CK(cudaGraphLaunch(h->g1[h->t % 6], h->stream));
            h->t++;
            n--;
        }
    }
    CK(cudaMemcpyAsync(h->h_err, h->sh.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(h->err_ev, h->stream));
    h->err_pending = true;
    return LB_OK;
}

int lb_sync(lb_handle* h) {
    if (!h) return LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    return read_err(h);
}

int lb_observables(lb_handle* h, int32_t box, lb_obs* out) {
    if (!h || !out || box < 0 || box >= h->nb) return LB_EINVAL;
    memset(out, 0, sizeof(*out));
    const BoxDev& B = h->hbox[box];
    cudaStream_t st = h->stream;
    const int par = (int)(h->t & 1);
    CK(h->ops->obs_partial(st, h->d_boxes, box, par, (int)(h->t % 3), h->obs_buf));
    double* fin = h->obs_buf + (size_t)OBS_BLOCKS * OBS_W;
    k_obs_final<<<1, 32, 0, st>>>(h->obs_buf, OBS_BLOCKS, fin);
    CK(cudaGetLastError());
    double v[OBS_W];
    CK(cudaMemcpyAsync(v, fin, sizeof(v), cudaMemcpyDeviceToHost, st));
    unsigned long long cnt[2];
    CK(cudaMemcpyAsync(cnt, h->sh.counters + 2 * box, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    std::vector<PartState> ps(B.np > 0 ? B.np : 1);
    if (B.np > 0)
        CK(cudaMemcpyAsync(ps.data(), h->sh.part + B.pstart, sizeof(PartState) * B.np, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->step = h->t;
    out->mass[0] = v[0];
    out->mass[1] = v[1];
    for (int a = 0; a < 3; a++) out->mom_fluid[a] = v[2 + a];
    out->max_u = v[5];
    out->n_fluid = (int64_t)v[6];
    out->n_solid = (int64_t)v[7];
    if (!h->params[box].fixed_particles)
        for (int q = 0; q < B.np; q++)
            for (int a = 0; a < 3; a++) out->mom_part[a] += B.mass * ps[q].U[a];
    out->n_cover = (int64_t)cnt[0];
    out->n_uncover = (int64_t)cnt[1];
    out->n_particles = B.np;
    int rc = structure_obs(h, box, out->L, &out->coverage, nullptr);
    if (rc != LB_OK) return rc;
    out->error = read_err(h);
    return LB_OK;
}

int lb_export_state(lb_handle* h, int32_t box, double* f, int32_t* owner, double* particles, double* meta) {
    if (!h || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    cudaStream_t st = h->stream;
    const int par = (int)(h->t & 1);
    CK(cudaStreamSynchronize(st));
    if (f) {
        // direction d (both components, 2N doubles) is converted into
        // staging slot d % 2 on the handle's stream and copied out on
        // xstream, so the conversion of d + 1 overlaps the copy of d
        const size_t N = (size_t)B.N;
        for (int d = 0; d < 19; d++) {
            const int k = d & 1;
            double* buf = h->stage + (size_t)k * 2 * N;
            if (d >= 2) CK(cudaStreamWaitEvent(st, h->ev_c[k], 0));
            CK(h->ops->export_dir(st, h->d_boxes, box, d, par, (int)(h->t % 3), buf));
            CK(cudaEventRecord(h->ev_k[k], st));
            CK(cudaStreamWaitEvent(h->xstream, h->ev_k[k], 0));
            for (int c = 0; c < 2; c++)
                CK(cudaMemcpyAsync(f + ((size_t)c * 19 + d) * N, buf + c * N, sizeof(double) * N,
                                   cudaMemcpyDeviceToHost, h->xstream));
            CK(cudaEventRecord(h->ev_c[k], h->xstream));
        }
        CK(cudaStreamSynchronize(h->xstream));
        CK(cudaStreamSynchronize(st));
    }
    if (owner) {
        // box-local particle indices, remapped on the device (staging
        // scratch) for every box after the first
        const int32_t* src = B.owner;
        if (B.pstart != 0) {
            int32_t* tmp = reinterpret_cast<int32_t*>(h->stage);
            k_owner_export<<<SMALL_GRID * 4, 256, 0, st>>>(B.owner, tmp, B.N, B.pstart);
            CK(cudaGetLastError());
            src = tmp;
        }
        CK(cudaMemcpyAsync(owner, src, sizeof(int32_t) * B.N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (particles && B.np > 0) {
        std::vector<PartState> ps(B.np);
        CK(cudaMemcpyAsync(ps.data(), h->sh.part + B.pstart, sizeof(PartState) * B.np, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int q = 0; q < B.np; q++)
            for (int a = 0; a < 3; a++) {
                particles[9 * q + a] = ps[q].X[a];
                particles[9 * q + 3 + a] = ps[q].U[a];
                particles[9 * q + 6 + a] = ps[q].W[a];
            }
    }
    if (meta) {
        meta[0] = (double)h->t;
        meta[1] = B.mass0[0];
        meta[2] = B.mass0[1];
        meta[3] = (double)B.np;
    }
    return LB_OK;
}

// The part of an import that both state formats share: the checks, the
// owner map (validated and remapped on the device before anything of the
// box changes), the particles, the node and shell flags.  The populations
// and densities are left to the caller.  *t_out: the step of the state.
static int import_begin(lb_handle* h, int32_t box, const int32_t* owner, const double* particles, const double* meta,
                        int64_t* t_out) {
    if (!owner || !meta) return LB_EINVAL;
    BoxDev& B = h->hbox[box];
    if (B.np > 0 && !particles) return LB_EINVAL;
    if ((int)meta[3] != B.np) return LB_EINVAL;
    const int64_t t = (int64_t)meta[0];
    if (t < 0) return LB_EINVAL;
    if (h->nb > 1 && h->initialised && t != h->t) return LB_EINVAL;
    cudaStream_t st = h->stream;
    const int N = B.N;
    {
        // validated and remapped on the device (scratch after the two
        // staging halves) before anything of the box changes; copied into the
        // box below, after the particles
        int32_t* raw = reinterpret_cast<int32_t*>(h->stage + 2 * (size_t)N);
        int32_t* mapped = raw + N;
        int* flags = reinterpret_cast<int*>(h->mass_tmp);
        int fl = 0;
        CK(cudaMemsetAsync(flags, 0, sizeof(int), st));
        CK(cudaMemcpyAsync(raw, owner, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
        k_owner_import<<<SMALL_GRID * 4, 256, 0, st>>>(raw, mapped, N, B.np, B.pstart, flags);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&fl, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (fl & 1) return LB_EINVAL;
        h->has_walls[box] = (fl & 2) ? 1 : 0;
    }
    if (B.np > 0) {
        std::vector<PartState> ps(B.np);
        std::vector<int> pb(B.np, box);
        std::vector<double> col(B.np, box_color(h->params[box]));
        // spheroid axes are not part of this format: a box that was stepped
        // keeps its current axes, otherwise those of the last lb_set_axes
        std::vector<double> ax = h->axes[box];
        if (h->initialised) {
            int rc = lb_get_axes(h, box, ax.data());
            if (rc != LB_OK) return rc;
        }
        for (int q = 0; q < B.np; q++)
            for (int a = 0; a < 3; a++) {
                ps[q].X[a] = particles[9 * q + a];
                ps[q].U[a] = particles[9 * q + 3 + a];
                ps[q].W[a] = particles[9 * q + 6 + a];
                ps[q].E[a] = ax[3 * q + a];
            }
        CK(cudaMemcpyAsync(h->sh.part + B.pstart, ps.data(), sizeof(PartState) * B.np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(h->sh.pbox + B.pstart, pb.data(), sizeof(int) * B.np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(h->sh.color + B.pstart, col.data(), sizeof(double) * B.np, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(h->sh.force + (size_t)B.pstart * 6, 0, sizeof(double) * 6 * B.np, st));
        CK(cudaMemsetAsync(h->sh.force_last + (size_t)B.pstart * 6, 0, sizeof(double) * 6 * B.np, st));
        k_part_to_float<<<(B.np + 255) / 256, 256, 0, st>>>(h->sh, B.pstart, B.np);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(B.owner, reinterpret_cast<int32_t*>(h->stage + 2 * (size_t)N) + N, sizeof(int32_t) * N,
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    B.mass0[0] = meta[1];
    B.mass0[1] = meta[2];
    fill_params(h);
    int rc = upload_boxes(h);
    if (rc != LB_OK) return rc;
    k_flags_from_owner<<<SMALL_GRID * 4, 256, 0, st>>>(h->d_boxes, box);
    k_shell_all<<<SMALL_GRID * 4, 256, 0, st>>>(h->d_boxes, box);
    CK(cudaGetLastError());
    *t_out = t;
    return LB_OK;
}

int lb_import_state(lb_handle* h, int32_t box, const double* f, const int32_t* owner, const double* particles,
                    const double* meta) {
    if (!h || box < 0 || box >= h->nb || !f) return LB_EINVAL;
    int64_t t = 0;
    int rc0 = import_begin(h, box, owner, particles, meta, &t);
    if (rc0 != LB_OK) return rc0;
    BoxDev& B = h->hbox[box];
    cudaStream_t st = h->stream;
    const int N = B.N;
    const int par = (int)(t & 1), rcs = (int)(t % 3);
    // direction d (both components, 2N doubles) is copied into staging slot
    // d % 2 on xstream and converted on the handle's stream, so the copy of
    // d + 1 overlaps the conversion of d (the owner scratch above is free
    // again: the map was copied into the box)
    CK(cudaEventRecord(h->ev_k[0], st));  // xstream starts after the work above
    CK(cudaStreamWaitEvent(h->xstream, h->ev_k[0], 0));
    for (int d = 0; d < 19; d++) {
        const int k = d & 1;
        double* buf = h->stage + (size_t)k * 2 * N;
        if (d >= 2) CK(cudaStreamWaitEvent(h->xstream, h->ev_k[k], 0));
        for (int c = 0; c < 2; c++)
            CK(cudaMemcpyAsync(buf + (size_t)c * N, f + ((size_t)c * 19 + d) * N, sizeof(double) * N,
                               cudaMemcpyHostToDevice, h->xstream));
        CK(cudaEventRecord(h->ev_c[k], h->xstream));
        CK(cudaStreamWaitEvent(st, h->ev_c[k], 0));
        CK(h->ops->import_dir(st, h->d_boxes, box, d, par, buf));
        CK(cudaEventRecord(h->ev_k[k], st));
    }
    for (int k = 0; k < 3; k++) CK(cudaMemsetAsync(B.rho[k], 0, (size_t)2 * N * h->ops->real_size, st));
    CK(cudaMemsetAsync(B.evmark, 0, sizeof(int32_t) * N, st));
    CK(cudaMemsetAsync(h->mass_tmp, 0, 2 * sizeof(double), st));
    CK(h->ops->rho_from_pop(st, h->d_boxes, box, par, -1, rcs, nullptr, h->mass_tmp));
    CK(cudaMemcpyAsync(B.mass_acc + 2 * par, h->mass_tmp, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(h->sh.counters + 2 * box, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(h->sh.err, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return after_init(h, t);
}

// Storage-format state of a box: the 18 stored population pairs of every
// node as the device holds them (slots 1..18 for FP64 / FP32 storage, after
// the rest slot that only an FP64-format import uses; the whole population
// array in 16-bit storage), then the density field of the current step.
static void native_layout(const lb_handle* h, const BoxDev& B, size_t* pop_off, size_t* pop_bytes,
                          size_t* rho_bytes) {
    const size_t N = (size_t)B.N, rs = h->ops->real_size;
    const bool dev = h->ops->id >= 2;
    *pop_off = dev ? 0 : 2 * N * rs;
    *pop_bytes = dev ? 2 * 18 * N * sizeof(uint16_t) : 2 * 18 * N * rs;
    *rho_bytes = 2 * N * rs;
}

int lb_state_native_bytes(lb_handle* h, int32_t box, size_t* bytes) {
    if (!h || !bytes || box < 0 || box >= h->nb) return LB_EINVAL;
    size_t po, pb, rb;
    native_layout(h, h->hbox[box], &po, &pb, &rb);
    *bytes = pb + rb;
    return LB_OK;
}

int lb_export_state_native(lb_handle* h, int32_t box, void* state, size_t bytes, int32_t* owner, double* particles,
                           double* meta) {
    if (!h || box < 0 || box >= h->nb) return LB_EINVAL;
    if (!h->initialised) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    size_t po, pb, rb;
    native_layout(h, B, &po, &pb, &rb);
    if (state && bytes != pb + rb) return LB_EINVAL;
    cudaStream_t st = h->stream;
    if (state) {
        CK(cudaMemcpyAsync(state, reinterpret_cast<const char*>(B.f) + po, pb, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(reinterpret_cast<char*>(state) + pb, B.rho[h->t % 3], rb, cudaMemcpyDeviceToHost, st));
    }
    double macc[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(macc, B.mass_acc + 2 * (h->t & 1), sizeof(macc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int rc = lb_export_state(h, box, nullptr, owner, particles, nullptr);
    if (rc != LB_OK) return rc;
    if (meta) {
        meta[0] = (double)h->t;
        meta[1] = B.mass0[0];
        meta[2] = B.mass0[1];
        meta[3] = (double)B.np;
        meta[4] = (double)h->ops->id;
        meta[5] = (double)B.N;
        meta[6] = macc[0];
        meta[7] = macc[1];
    }
    return LB_OK;
}

int lb_import_state_native(lb_handle* h, int32_t box, const void* state, size_t bytes, const int32_t* owner,
                           const double* particles, const double* meta) {
    if (!h || box < 0 || box >= h->nb || !state || !meta) return LB_EINVAL;
    BoxDev& B = h->hbox[box];
    size_t po, pb, rb;
    native_layout(h, B, &po, &pb, &rb);
    if (bytes != pb + rb || (int)meta[4] != h->ops->id || (int64_t)meta[5] != (int64_t)B.N) return LB_EINVAL;
    int64_t t = 0;
    int rc0 = import_begin(h, box, owner, particles, meta, &t);
    if (rc0 != LB_OK) return rc0;
    cudaStream_t st = h->stream;
    const int par = (int)(t & 1), rcs = (int)(t % 3);
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(B.f) + po, state, pb, cudaMemcpyHostToDevice, st));
    // the ring slots of the next steps start zeroed (the fused kernel adds
    // into the nodes at tile edges of the slot it fills)
    for (int k = 0; k < 3; k++) CK(cudaMemsetAsync(B.rho[k], 0, rb, st));
    CK(cudaMemcpyAsync(B.rho[rcs], reinterpret_cast<const char*>(state) + pb, rb, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(B.evmark, 0, sizeof(int32_t) * B.N, st));
    CK(cudaMemcpyAsync(B.mass_acc + 2 * par, meta + 6, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(h->sh.counters + 2 * box, 0, 2 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(h->sh.err, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return after_init(h, t);
}

int lb_export_rho(lb_handle* h, int32_t box, double* rho) {
    if (!h || !rho || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    cudaStream_t st = h->stream;
    CK(h->ops->rho_from_pop(st, h->d_boxes, box, (int)(h->t & 1), (int)(h->t % 3), -1, h->stage, nullptr));
    CK(cudaMemcpyAsync(rho, h->stage, sizeof(double) * 2 * B.N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return LB_OK;
}

int lb_export_phi(lb_handle* h, int32_t box, double* phi, double L[3], double* coverage) {
    if (!h || box < 0 || box >= h->nb) return LB_EINVAL;
    if (!h->initialised) return LB_EINVAL;
    double Ld[3], cov;
    int rc = structure_obs(h, box, Ld, &cov, phi);
    if (rc != LB_OK) return rc;
    if (L)
        for (int a = 0; a < 3; a++) L[a] = Ld[a];
    if (coverage) *coverage = cov;
    return LB_OK;
}

int lb_set_particle_colors(lb_handle* h, int32_t box, const double* colors) {
    if (!h || !colors || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    if (B.np == 0) return LB_OK;
    CK(cudaMemcpyAsync(h->sh.color + B.pstart, colors, sizeof(double) * B.np, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_set_axes(lb_handle* h, int32_t box, const double* e) {
    if (!h || !e || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    if (B.np == 0) return LB_OK;
    std::vector<double> v((size_t)3 * B.np);
    for (int q = 0; q < B.np; q++) {
        const double n = std::sqrt(e[3 * q] * e[3 * q] + e[3 * q + 1] * e[3 * q + 1] + e[3 * q + 2] * e[3 * q + 2]);
        if (!(std::fabs(n - 1.0) < 1e-6)) return LB_EINVAL;
        for (int a = 0; a < 3; a++) v[3 * q + a] = e[3 * q + a];
    }
    h->axes[box] = v;
    // the device copy (strided into the particle records)
    CK(cudaMemcpy2DAsync(reinterpret_cast<char*>(h->sh.part + B.pstart) + offsetof(PartState, E), sizeof(PartState),
                         v.data(), 3 * sizeof(double), 3 * sizeof(double), B.np, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_get_axes(lb_handle* h, int32_t box, double* e) {
    if (!h || !e || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    if (B.np == 0) return LB_OK;
    CK(cudaMemcpy2DAsync(e, 3 * sizeof(double), reinterpret_cast<const char*>(h->sh.part + B.pstart) + offsetof(PartState, E),
                         sizeof(PartState), 3 * sizeof(double), B.np, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb_particle_forces(lb_handle* h, int32_t box, double* F, double* T) {
    if (!h || box < 0 || box >= h->nb) return LB_EINVAL;
    const BoxDev& B = h->hbox[box];
    if (B.np == 0) return LB_OK;
    std::vector<double> v((size_t)B.np * 6);
    CK(cudaMemcpyAsync(v.data(), h->sh.force_last + (size_t)B.pstart * 6, sizeof(double) * 6 * B.np,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int q = 0; q < B.np; q++)
        for (int a = 0; a < 3; a++) {
            if (F) F[3 * q + a] = v[6 * q + a];
            if (T) T[3 * q + a] = v[6 * q + 3 + a];
        }
    return LB_OK;
}

int lb_box_info(lb_handle* h, int32_t box, int32_t* n_particles, int64_t* n_nodes) {
    if (!h || box < 0 || box >= h->nb) return LB_EINVAL;
    if (n_particles) *n_particles = h->hbox[box].np;
    if (n_nodes) *n_nodes = h->hbox[box].N;
    return LB_OK;
}

int lb_set_tiling(lb_handle* h, int32_t ty, int32_t cz, int32_t split) {
    if (!h || cz < 1 || (split != 0 && split != 1)) return LB_EINVAL;
    if (split ? (ty != 8 && ty != 16) : (ty != 4 && ty != 8 && ty != 16)) return LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    h->ty = ty;
    h->cz = cz;
    h->split = split;
    int rc = build_tiles(h);
    if (rc != LB_OK) return rc;
    // The next step adds into its density buffer at the new tiling's edge
    // nodes, which the previous step only zeroed for the old tiling.
    if (h->initialised) {
        for (int b = 0; b < h->nb; b++)
            CK(cudaMemsetAsync(h->hbox[b].rho[(h->t + 1) % 3], 0, (size_t)2 * h->hbox[b].N * h->ops->real_size,
                               h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    destroy_graphs(h);
    if (h->initialised && h->stream) return build_graphs(h);
    return LB_OK;
}

int lb_set_profiling(lb_handle* h, int32_t on) {
    if (!h) return LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    h->prof = on != 0;
    h->ev_used = 0;
    h->phase_marks.clear();
    h->prof_ms = 0.0;
    h->prof_fused = 0;
    h->prof_total = 0;
    return LB_OK;
}

int lb_kernel_time(lb_handle* h, double* ms_fused, int64_t* launches_fused, int64_t* launches_total) {
    if (!h) return LB_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    // phase k of a step lasts from its mark to the next mark of the step
    for (int k = 0; k < LB_NPHASES; k++) h->phase_ms[k] = 0.0;
    for (size_t k = 0; k + 1 < h->phase_marks.size(); k++) {
        const int ph = h->phase_marks[k].first;
        if (ph >= LB_NPHASES) continue;  // end-of-step mark
        float v = 0.f;
        CK(cudaEventElapsedTime(&v, h->evpool[h->phase_marks[k].second], h->evpool[h->phase_marks[k + 1].second]));
        h->phase_ms[ph] += v;
    }
    h->phase_marks.clear();
    if (ms_fused) *ms_fused = h->phase_ms[4];
    if (launches_fused) *launches_fused = h->prof_fused;
    if (launches_total) *launches_total = h->prof_total;
    h->ev_used = 0;
    h->prof_fused = 0;
    h->prof_total = 0;
    return LB_OK;
}

int lb_phase_times(lb_handle* h, double* ms, int32_t n) {
    if (!h || !ms || n < 0) return LB_EINVAL;
    for (int k = 0; k < n && k < LB_NPHASES; k++) ms[k] = h->phase_ms[k];
    return LB_OK;
}

void lb_destroy(lb_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    for (auto e : h->evpool) cudaEventDestroy(e);
    if (h->err_ev) cudaEventDestroy(h->err_ev);
    if (h->xstream) {
        cudaStreamSynchronize(h->xstream);
        cudaStreamDestroy(h->xstream);
    }
    for (int b = 0; b < 2; b++) {
        if (h->ev_k[b]) cudaEventDestroy(h->ev_k[b]);
        if (h->ev_c[b]) cudaEventDestroy(h->ev_c[b]);
    }
    if (h->mdstream) {
        cudaStreamSynchronize(h->mdstream);
        cudaStreamDestroy(h->mdstream);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->h_err) cudaFreeHost(h->h_err);
    delete h;
}

}  // extern "C"
