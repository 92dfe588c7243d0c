// C-ABI of libpond (declared in include/pond.h): configuration checks, workspace layout,
// the time-step loop and host <-> device transfers.  No device memory is allocated here:
// the caller provides the workspace.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "pond.h"
#include "pond_aux.cuh"
#include "pond_launch.h"
#include "pond_step.cuh"

using namespace pond;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t storage_bytes(int precision)
{
    switch (precision) {
        case POND_FP64: return 8;
        case POND_MIXED_FP32: return 4;
        default: return 2;
    }
}

// Table I quadratures (Gauss-Hermite, r T_L = 1) and the derived Hermite values.
Lattice make_lattice(int q1)
{
    Lattice L;
    std::memset(&L, 0, sizeof(L));
    L.q1 = q1;
    if (q1 == 4) {
        const double ci = std::sqrt(3.0 - std::sqrt(6.0)), co = std::sqrt(3.0 + std::sqrt(6.0));
        const double wi = (3.0 + std::sqrt(6.0)) / 12.0, wo = (3.0 - std::sqrt(6.0)) / 12.0;
        const double c[4] = {-co, -ci, ci, co}, w[4] = {wo, wi, wi, wo};
        for (int a = 0; a < 4; ++a) { L.c[a] = c[a]; L.w[a] = w[a]; }
        L.cmax = co;
    } else {
        const double ci = std::sqrt(5.0 - std::sqrt(10.0)), co = std::sqrt(5.0 + std::sqrt(10.0));
        const double w0 = 8.0 / 15.0, wi = (7.0 + 2.0 * std::sqrt(10.0)) / 60.0;
        const double wo = (7.0 - 2.0 * std::sqrt(10.0)) / 60.0;
        const double c[5] = {-co, -ci, 0.0, ci, co}, w[5] = {wo, wi, w0, wi, wo};
        for (int a = 0; a < 5; ++a) { L.c[a] = c[a]; L.w[a] = w[a]; }
        L.cmax = co;
    }
    L.cmaxf = (float)L.cmax;
    const double fact[5] = {1.0, 1.0, 2.0, 6.0, 24.0};
    for (int a = 0; a < q1; ++a) {
        const double x = L.c[a];
        const double he[5] = {1.0, x, x * x - 1.0, x * x * x - 3.0 * x, x * x * x * x - 6.0 * x * x + 3.0};
        for (int p = 0; p < 5; ++p) {
            L.he[a][p] = he[p];
            L.hn[a][p] = he[p] / fact[p];
            L.hef[a][p] = (float)L.he[a][p];
            L.hnf[a][p] = (float)L.hn[a][p];
        }
        L.cf[a] = (float)L.c[a];
        L.wf[a] = (float)L.w[a];
    }
    return L;
}

struct Layout {
    size_t mac[2], neq[2], status, prof[4], total;   // prof[side] = 0: the side takes no profile
    size_t upred;                                    // internal split: predictor region (upred_bytes); else 0
};

// Grad order of a configuration: the lattice's (3 on D2Q16, 4 on D2Q25).
int grad_order(const pond_config& c) { return c.lattice == POND_D2Q25 ? 4 : 3; }

// Whether side w (0 x-low, 1 x-high, 2 y-low, 3 y-high) is prescribed: both sides of a wall
// axis, the low side of an inflow axis.
bool side_prescribed(const pond_config& c, int w)
{
    const int bc = w < 2 ? c.bc_x : c.bc_y;
    return bc == POND_BC_WALL || (bc == POND_BC_INFLOW && (w % 2) == 0);
}

// Positions along side w: ny for the x sides, nx for the y sides.
int side_length(const pond_config& c, int w) { return w < 2 ? c.ny : c.nx; }

// Bytes of the internal split's predictor region: the predictor velocities, [2][N] doubles,
// followed by the coefficients of the populations it streamed, [2 ncoef][N] values of the
// arithmetic type (double in the FP64 mode, float otherwise).
size_t upred_bytes(const pond_config& c)
{
    const size_t N = (size_t)c.nx * (size_t)c.ny;
    const size_t nc = (size_t)ncoef(grad_order(c));
    return 2 * N * sizeof(double) + 2 * nc * N * (c.precision == POND_FP64 ? sizeof(double) : sizeof(float));
}

Layout layout_of(const pond_config& c)
{
    const size_t N = (size_t)c.nx * (size_t)c.ny;
    const size_t planes = (size_t)nneq(grad_order(c));
    Layout l;
    size_t off = 0;
    for (int k = 0; k < 2; ++k) { l.mac[k] = off; off = align_up(off + NMAC * N * sizeof(double)); }
    for (int k = 0; k < 2; ++k) { l.neq[k] = off; off = align_up(off + planes * N * storage_bytes(c.precision)); }
    l.status = off;
    off = align_up(off + sizeof(DevStatus));
    for (int w = 0; w < 4; ++w) {
        l.prof[w] = 0;
        if (!side_prescribed(c, w)) continue;
        l.prof[w] = off;
        off = align_up(off + 4 * (size_t)side_length(c, w) * sizeof(double));
    }
    l.upred = 0;
    if (c.split == POND_SPLIT_INTERNAL) {
        l.upred = off;
        off = align_up(off + upred_bytes(c));
    }
    l.total = off;
    return l;
}

int check_config(const pond_config* c)
{
    if (!c) return POND_EINVAL;
    if (c->nx < 1 || c->ny < 1) return POND_EINVAL;
    if ((long long)c->nx * (long long)c->ny > (1ll << 31)) return POND_EINVAL;
    if (c->lattice != POND_D2Q16 && c->lattice != POND_D2Q25) return POND_EINVAL;
    if (c->split != POND_SPLIT_TOTAL && c->split != POND_SPLIT_INTERNAL && c->split != POND_SPLIT_NT)
        return POND_EINVAL;
    // the Grad order is the lattice's: 3 on D2Q16, 4 on D2Q25
    if (c->grad_order != 0 && c->grad_order != (c->lattice == POND_D2Q25 ? 4 : 3)) return POND_EINVAL;
    if (c->precision < POND_FP64 || c->precision > POND_MIXED_BF16) return POND_EINVAL;
    if (c->interp_order != 2 && c->interp_order != 3) return POND_EINVAL;
    if (c->bc_x < 0 || c->bc_x > 3 || c->bc_y < 0 || c->bc_y > 3) return POND_EINVAL;
    // quasi-1-D grids have no prescribed y sides
    if ((c->bc_y == POND_BC_WALL || c->bc_y == POND_BC_INFLOW) && c->ny == 1) return POND_EINVAL;
    for (int w = 0; w < 4; ++w) {
        const bool used = side_prescribed(*c, w);
        const double* st = c->wall[w];
        if (used && !(st[2] > 0.0 && st[3] > 0.0 && std::isfinite(st[0]) && std::isfinite(st[1]) &&
                      std::isfinite(st[2]) && std::isfinite(st[3])))
            return POND_EINVAL;
    }
    if (!(c->gamma > 1.0 && c->gamma <= 2.0)) return POND_EINVAL;   // U' >= 0 in 2-D needs gamma <= 2
    if (!(c->mu > 0.0) || !std::isfinite(c->mu)) return POND_EINVAL;
    if (!(c->pc_tol >= 0.0)) return POND_EINVAL;
    if (c->pc_max_iter < 1 || c->pc_max_iter > 64) return POND_EINVAL;
    if (c->pc_fixed_iters < 0 || c->pc_fixed_iters > 64) return POND_EINVAL;
    if (c->tile_x < 0 || c->tile_y < 0 || c->halo < 0 || c->halo > 64) return POND_EINVAL;
    if (c->tile_x || c->tile_y) {
        int t = c->tile_x * c->tile_y;
        if (c->tile_x < 1 || c->tile_y < 1 || t != step_threads(c->ny == 1)) return POND_EINVAL;
        if (c->ny == 1 && c->tile_y != 1) return POND_EINVAL;
    }
    return POND_OK;
}

}  // namespace

struct pond_sim {
    pond_config cfg;
    cudaStream_t stream;
    char* ws;
    Layout lay;
    int cur;
    long long steps;
    Lattice lat;
    int tx, ty, box_w, box_h;
    size_t smem;
    bool one_d;
    DevStatus host_status;
};

namespace {

double* mac_ptr(pond_sim* s, int k) { return reinterpret_cast<double*>(s->ws + s->lay.mac[k]); }
void* neq_ptr(pond_sim* s, int k) { return s->ws + s->lay.neq[k]; }
DevStatus* status_ptr(pond_sim* s) { return reinterpret_cast<DevStatus*>(s->ws + s->lay.status); }
double* prof_ptr(pond_sim* s, int w) { return reinterpret_cast<double*>(s->ws + s->lay.prof[w]); }
double* upred_ptr(pond_sim* s) { return s->lay.upred ? reinterpret_cast<double*>(s->ws + s->lay.upred) : nullptr; }

// The profiles a simulation's kernels read: every prescribed side streams from its profile in
// the workspace (filled with the side's uniform state at creation); null for the other sides.
void side_profiles(pond_sim* s, const double* prof[4])
{
    for (int w = 0; w < 4; ++w) prof[w] = s->lay.prof[w] ? prof_ptr(s, w) : nullptr;
}

int cuda_status(cudaError_t e);

// Blocks of the step kernel resident at once on the current device (step_blocks_per_sm per
// SM: the distance of the next-wave L2 prefetch).  0 if the query fails.
int resident_step_blocks(const pond_config& c, bool one_d)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * step_blocks_per_sm(one_d, c.lattice == POND_D2Q25, c.precision == POND_FP64);
}

// Copy states [n][4] (host or device) into side w's profile, or its uniform state when
// state is null.  Host states are checked (T > 0, rho > 0, finite).
int write_profile(pond_sim* s, int w, const double* state, int on_device)
{
    const int n = side_length(s->cfg, w);
    const size_t nb = 4 * (size_t)n * sizeof(double);
    cudaError_t e;
    if (state && on_device) {
        e = cudaMemcpyAsync(prof_ptr(s, w), state, nb, cudaMemcpyDeviceToDevice, s->stream);
    } else {
        std::vector<double> h(4 * (size_t)n);
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < 4; ++j) h[4 * (size_t)k + j] = state ? state[4 * (size_t)k + j] : s->cfg.wall[w][j];
        for (int k = 0; k < n; ++k) {
            const double* st = &h[4 * (size_t)k];
            if (!(st[2] > 0.0 && st[3] > 0.0 && std::isfinite(st[0]) && std::isfinite(st[1]) &&
                  std::isfinite(st[2]) && std::isfinite(st[3])))
                return POND_EINVAL;
        }
        // pageable source: the copy has read it when the call returns
        e = cudaMemcpyAsync(prof_ptr(s, w), h.data(), nb, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    return cuda_status(e);
}

AuxParams aux_params(pond_sim* s, int k)
{
    AuxParams a;
    std::memset(&a, 0, sizeof(a));
    a.lat = s->lat;
    a.nx = s->cfg.nx;
    a.ny = s->cfg.ny;
    a.bc_x = s->cfg.bc_x;
    a.bc_y = s->cfg.bc_y;
    a.split = s->cfg.split;
    a.nord = grad_order(s->cfg);
    std::memcpy(a.wall, s->cfg.wall, sizeof(a.wall));
    side_profiles(s, a.prof);
    a.N = (long long)s->cfg.nx * s->cfg.ny;
    a.cv = 1.0 / (s->cfg.gamma - 1.0);
    a.mu = s->cfg.mu;
    a.mac = mac_ptr(s, k);
    a.neq = neq_ptr(s, k);
    a.mac_prev = mac_ptr(s, 1 - k);
    a.status = status_ptr(s);
    return a;
}

#define POND_BY_PRECISION(prec, FN, ...)                                  \
    ((prec) == POND_FP64 ? FN##_f64(__VA_ARGS__)                          \
     : (prec) == POND_MIXED_FP32 ? FN##_f32(__VA_ARGS__)                  \
     : (prec) == POND_MIXED_FP16 ? FN##_f16(__VA_ARGS__) : FN##_bf16(__VA_ARGS__))

// Step launchers indexed [precision][q1 == 5][one_d].
const StepFn kStep[4][2][2] = {
    {{step_f64_q4_2d, step_f64_q4_1d}, {step_f64_q5_2d, step_f64_q5_1d}},
    {{step_f32_q4_2d, step_f32_q4_1d}, {step_f32_q5_2d, step_f32_q5_1d}},
    {{step_f16_q4_2d, step_f16_q4_1d}, {step_f16_q5_2d, step_f16_q5_1d}},
    {{step_bf16_q4_2d, step_bf16_q4_1d}, {step_bf16_q5_2d, step_bf16_q5_1d}},
};
const SmemFn kSmem[4][2][2] = {
    {{smem_f64_q4_2d, smem_f64_q4_1d}, {smem_f64_q5_2d, smem_f64_q5_1d}},
    {{smem_f32_q4_2d, smem_f32_q4_1d}, {smem_f32_q5_2d, smem_f32_q5_1d}},
    {{smem_f16_q4_2d, smem_f16_q4_1d}, {smem_f16_q5_2d, smem_f16_q5_1d}},
    {{smem_bf16_q4_2d, smem_bf16_q4_1d}, {smem_bf16_q5_2d, smem_bf16_q5_1d}},
};

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return POND_OK;
    std::fprintf(stderr, "libpond: CUDA error %s\n", cudaGetErrorString(e));
    return POND_ECUDA;
}

// Zero the status block (first_bad = ~0: none), on the stream, without a host copy.
int reset_status(pond_sim* s)
{
    s->steps = 0;
    DevStatus* st = status_ptr(s);
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st->first_bad, 0xff, sizeof(st->first_bad), s->stream);
    return cuda_status(e);
}

// Page-locked mirror of a status block for the synchronising reads of this host thread
// (a copy into pageable memory goes through a staging buffer and costs several times a
// small pinned copy).  Allocated at the thread's first synchronising call and kept; null
// if the allocation failed, and the reads then go to pageable memory.
DevStatus* pinned_status_mirror()
{
    static thread_local DevStatus* mirror = nullptr;
    static thread_local bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        if (cudaMallocHost(&p, sizeof(DevStatus)) == cudaSuccess) mirror = static_cast<DevStatus*>(p);
        else cudaGetLastError();
    }
    return mirror;
}

// Copy the status block to s->host_status and synchronise the stream.
cudaError_t read_status(pond_sim* s)
{
    DevStatus* m = pinned_status_mirror();
    DevStatus* dst = m ? m : &s->host_status;
    cudaError_t e = cudaMemcpyAsync(dst, status_ptr(s), sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess && m) std::memcpy(&s->host_status, m, sizeof(DevStatus));
    return e;
}

// Synchronise and translate the sticky device status.
int sync_status(pond_sim* s)
{
    cudaError_t e = read_status(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->host_status.flags & 1) return POND_ENONPHYSICAL;
    if (s->host_status.flags & 2) return POND_ENOCONV;
    return POND_OK;
}

// Parameters of one case for the step kernel (buffers filled by the caller); prof: the
// sides' profiles (null: uniform states).
void fill_case(const pond_config& c, DevStatus* status, CaseDesc& d, const double* const* prof = nullptr)
{
    std::memset(&d, 0, sizeof(d));
    d.nx = c.nx;
    d.ny = c.ny;
    d.bc_x = c.bc_x;
    d.bc_y = c.bc_y;
    d.split = c.split;
    d.nord = grad_order(c);
    d.pc_max_iter = c.pc_max_iter;
    d.pc_fixed = c.pc_fixed_iters;
    d.N = (long long)c.nx * c.ny;
    d.cv = 1.0 / (c.gamma - 1.0);
    d.inv_cv = c.gamma - 1.0;
    d.mu = c.mu;
    d.pc_tol = c.pc_tol;
    d.cv_f = (float)d.cv;
    d.inv_cv_f = (float)d.inv_cv;
    d.mu_f = (float)d.mu;
    d.pc_tol_f = (float)d.pc_tol;
    d.cur = 0;
    d.status = status;
    std::memcpy(d.wall, c.wall, sizeof(d.wall));
    for (int w = 0; w < 4; ++w) d.prof[w] = prof ? prof[w] : nullptr;
}

// Launch shape of the step kernel: the tile (tile_x * tile_y nodes per CTA; 0 = default,
// 32 x 8 on 2-D grids, 128 x 1 on quasi-1-D ones) and the staged box, the tile plus
// 2 halo + 2 cells per axis (halo 0 = default 5).
struct Shape {
    int tx, ty, box_w, box_h, halo;
    size_t smem;
    bool one_d;
};

int make_shape(const pond_config& c, int tile_x, int tile_y, int halo, Shape* sh)
{
    if (tile_x < 0 || tile_y < 0 || halo < 0 || halo > 64) return POND_EINVAL;
    sh->one_d = (c.ny == 1);
    if (sh->one_d) {
        if ((tile_x && tile_x != kStepThreads1D) || (tile_y && tile_y != 1)) return POND_EINVAL;
        sh->tx = kStepThreads1D;
        sh->ty = 1;
    } else {
        if ((tile_x != 0) != (tile_y != 0)) return POND_EINVAL;
        sh->tx = tile_x ? tile_x : 32;
        sh->ty = tile_y ? tile_y : kStepThreads2D / 32;
        if (sh->tx * sh->ty != kStepThreads2D || sh->tx % 2) return POND_EINVAL;
    }
    sh->halo = halo ? halo : 5;
    const int extent = 2 * sh->halo + 2;
    sh->box_w = sh->tx + extent;
    sh->box_h = sh->one_d ? 1 : sh->ty + extent;
    const int q1 = c.lattice == POND_D2Q16 ? 4 : 5;
    sh->smem = step_smem_bytes(c.precision == POND_FP64 ? 8 : 4, q1, sh->one_d, sh->box_w, sh->box_h,
                               step_threads(sh->one_d));
    int dev = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_status(e);
    // The limit is an attribute of the kernel, shared by every simulation of the process: set
    // it to the device's largest (less the kernel's static part), never to this shape's need,
    // so that a smaller shape set later cannot shrink it under a larger one.
    size_t static_bytes = 0;
    e = kSmem[c.precision][q1 == 5][sh->one_d](c.interp_order, (size_t)smem_optin, &static_bytes);
    if (e != cudaSuccess) return cuda_status(e);
    if (sh->smem + static_bytes > (size_t)smem_optin) return POND_EINVAL;   // box too large: lower halo or tile
    return POND_OK;
}

int apply_shape(pond_sim* s, int tile_x, int tile_y, int halo)
{
    Shape sh;
    int rc = make_shape(s->cfg, tile_x, tile_y, halo, &sh);
    if (rc != POND_OK) return rc;
    s->one_d = sh.one_d;
    s->tx = sh.tx;
    s->ty = sh.ty;
    s->box_w = sh.box_w;
    s->box_h = sh.box_h;
    s->smem = sh.smem;
    s->cfg.tile_x = s->one_d ? 0 : sh.tx;
    s->cfg.tile_y = s->one_d ? 0 : sh.ty;
    s->cfg.halo = sh.halo;
    return POND_OK;
}

}  // namespace

extern "C" {

const char* pond_version(void) { return "libpond 0.1 (sm_103a)"; }

const char* pond_strerror(int status)
{
    switch (status) {
        case POND_OK: return "ok";
        case POND_EINVAL: return "invalid argument or configuration";
        case POND_ENOMEM: return "workspace too small";
        case POND_ECUDA: return "CUDA runtime error";
        case POND_ENONPHYSICAL: return "non-physical state (rho <= 0, T <= 0 or NaN)";
        case POND_ENOCONV: return "predictor-corrector did not converge at some node";
        default: return "unknown status";
    }
}

int pond_config_default(pond_config* cfg, int32_t nx, int32_t ny)
{
    if (!cfg) return POND_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = nx;
    cfg->ny = ny;
    cfg->lattice = POND_D2Q16;
    cfg->split = POND_SPLIT_TOTAL;
    cfg->precision = POND_MIXED_FP32;
    cfg->interp_order = 3;
    cfg->bc_x = POND_BC_PERIODIC;
    cfg->bc_y = POND_BC_PERIODIC;
    cfg->gamma = 1.4;
    cfg->mu = 1e-3;
    cfg->pc_tol = 1e-6;
    cfg->pc_max_iter = 20;
    cfg->pc_fixed_iters = 0;
    return check_config(cfg);
}

int pond_workspace_bytes(const pond_config* cfg, size_t* bytes)
{
    int rc = check_config(cfg);
    if (rc != POND_OK) return rc;
    if (!bytes) return POND_EINVAL;
    *bytes = layout_of(*cfg).total;
    return POND_OK;
}

int pond_create(const pond_config* cfg, void* dev_workspace, size_t bytes, void* cuda_stream,
                pond_sim** out)
{
    if (!out) return POND_EINVAL;
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc != POND_OK) return rc;
    if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign)) return POND_EINVAL;
    Layout lay = layout_of(*cfg);
    if (bytes < lay.total) return POND_ENOMEM;
    pond_sim* s = new (std::nothrow) pond_sim;
    if (!s) return POND_ENOMEM;
    std::memset(s, 0, sizeof(*s));
    s->cfg = *cfg;
    s->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    s->ws = reinterpret_cast<char*>(dev_workspace);
    s->lay = lay;
    s->cur = 0;
    s->lat = make_lattice(cfg->lattice == POND_D2Q16 ? 4 : 5);
    rc = apply_shape(s, cfg->tile_x, cfg->tile_y, cfg->halo);
    if (rc != POND_OK) {
        delete s;
        return rc;
    }
    cudaError_t e = cudaSuccess;
    {
        rc = reset_status(s);
        if (rc != POND_OK) { delete s; return rc; }
        e = cudaMemsetAsync(s->ws, 0, lay.status, s->stream);
    }
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e);
    }
    for (int w = 0; w < 4; ++w) {   // prescribed sides start from their uniform states
        if (!lay.prof[w]) continue;
        rc = write_profile(s, w, nullptr, 0);
        if (rc != POND_OK) { delete s; return rc; }
    }
    *out = s;
    return POND_OK;
}

int pond_set_boundary_profile(pond_sim* s, int32_t side, const double* state, int on_device)
{
    if (!s || side < 0 || side > 3) return POND_EINVAL;
    if (!s->lay.prof[side]) return POND_EINVAL;   // the side is not prescribed
    return write_profile(s, side, state, on_device);
}

// Host input of pond_set_state, staged on the device: sets kInputBad when a node has rho <= 0, T <= 0 or a value that is not finite.  One flag
// write per warp.
__device__ __forceinline__ bool bad_fields(double r, double ux, double uy, double t)
{
    return !(r > 0.0) || !(t > 0.0) || !isfinite(r) || !isfinite(t) || !isfinite(ux) || !isfinite(uy);
}

__global__ void check_fields_kernel(const double* rho, const double* vx, const double* vy, const double* T,
                                    long long N, DevStatus* st)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = n < N && bad_fields(rho[n], vx[n], vy[n], T[n]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->flags, kInputBad);
}

// Batched form over members [c0, c1) of a batch (blocks from block_start[c0] = block0 on; a block
// lies within one member): the fields of member c are fld.f[c - c0].
__global__ void check_fields_batch_kernel(const CaseDesc* cases, const int* block_start, int c0, int c1,
                                          int block0, MemberFields fld)
{
    const int b = block0 + (int)blockIdx.x;
    const int c = member_of_block(block_start, c0, c1, b);
    const CaseDesc& d = cases[c];
    const long long n = (long long)(b - block_start[c]) * blockDim.x + threadIdx.x;
    const double* const* in = fld.f[c - c0];
    const bool bad = n < d.N && bad_fields(in[0][n], in[1][n], in[2][n], in[3][n]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&d.status->flags, kInputBad);
}

// Page-locked host input of members [c0, c1) (fld.f[c - c0]: device addresses of the host
// arrays) read in place, checked like check_fields_batch_kernel and written into the member's
// idle state buffer (cur ^ flip ^ 1), where the init kernel then reads it.
__global__ void stage_check_batch_kernel(const CaseDesc* cases, const int* block_start, int c0, int c1,
                                         int block0, int flip, MemberFields fld)
{
    const int b = block0 + (int)blockIdx.x;
    const int c = member_of_block(block_start, c0, c1, b);
    const CaseDesc& d = cases[c];
    const long long n = (long long)(b - block_start[c]) * blockDim.x + threadIdx.x;
    bool bad = false;
    if (n < d.N) {
        const double* const* in = fld.f[c - c0];
        const double r = in[0][n], ux = in[1][n], uy = in[2][n], t = in[3][n];
        double* stage = d.mac[d.cur ^ flip ^ 1];
        stage[n] = r;
        stage[d.N + n] = ux;
        stage[2 * d.N + n] = uy;
        stage[3 * d.N + n] = t;
        bad = bad_fields(r, ux, uy, t);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&d.status->flags, kInputBad);
}

// The status blocks of a batch's members cleared as reset_status clears one (first_bad = ~0).
__global__ void reset_status_batch_kernel(const CaseDesc* cases, int count)
{
    const int c = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= count) return;
    DevStatus* st = cases[c].status;
    *st = DevStatus{};
    st->first_bad = ~0ull;
}

// The device address of page-locked host memory (kernels then read or write it directly,
// without a staging copy), or null for any other host memory.
const double* host_view(const double* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const double*>(a.devicePointer) : nullptr;
}

// Device views of four host fields, all or none (null entries stay null).
bool host_views(const double* const in[4], const double* out[4])
{
    for (int k = 0; k < 4; ++k) {
        out[k] = nullptr;
        if (!in[k]) continue;
        out[k] = host_view(in[k]);
        if (!out[k]) return false;
    }
    return true;
}

int pond_set_state(pond_sim* s, const double* rho, const double* ux, const double* uy, const double* T,
                   int on_device)
{
    if (!s || !rho || !ux || !uy || !T) return POND_EINVAL;
    const long long N = (long long)s->cfg.nx * s->cfg.ny;
    int rc = reset_status(s);
    if (rc != POND_OK) return rc;
    AuxParams a = aux_params(s, s->cur);
    if (on_device)
        return cuda_status(POND_BY_PRECISION(s->cfg.precision, init, a, rho, ux, uy, T, s->stream));
    // Host input is copied into the idle frame buffer (one DMA copy per field: reading
    // page-locked memory in place from both the check and the initialisation saved only
    // about 5 % of this call, for four batched 256^2 grids) and
    // checked there on the device (the host's single core would take far longer over the same
    // bytes than the copy); the initialisation skips a rejected input, and one synchronisation
    // returns the outcome.
    const double* in[4] = {rho, ux, uy, T};
    const double* src[4];
    double* stage = mac_ptr(s, 1 - s->cur);
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = cudaMemcpyAsync(stage + k * N, in[k], N * sizeof(double), cudaMemcpyHostToDevice,
                                        s->stream);
        if (e != cudaSuccess) return cuda_status(e);
        src[k] = stage + k * N;
    }
    check_fields_kernel<<<(unsigned int)((N + 255) / 256), 256, 0, s->stream>>>(src[0], src[1], src[2], src[3],
                                                                              N, status_ptr(s));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = POND_BY_PRECISION(s->cfg.precision, init, a, src[0], src[1], src[2], src[3], s->stream);
    if (e == cudaSuccess) e = read_status(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (s->host_status.flags & kInputBad) {
        rc = reset_status(s);
        return rc != POND_OK ? rc : POND_EINVAL;
    }
    return POND_OK;
}

int pond_set_populations(pond_sim* s, const double* f, const double* g, const double* ux, const double* uy,
                         const double* T, int on_device)
{
    if (!s || !f || !g || !ux || !uy || !T) return POND_EINVAL;
    if (!on_device) return POND_EINVAL;   // populations move through device buffers only
    int rc = reset_status(s);
    if (rc != POND_OK) return rc;
    AuxParams a = aux_params(s, s->cur);
    return cuda_status(POND_BY_PRECISION(s->cfg.precision, set_pops, a, f, g, ux, uy, T, s->stream));
}

int pond_step(pond_sim* s, int32_t nsteps)
{
    if (!s || nsteps < 0) return POND_EINVAL;
    const pond_config& c = s->cfg;
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.lat = s->lat;
    p.box_w = s->box_w;
    p.box_h = s->box_h;
    p.ahead = resident_step_blocks(s->cfg, s->one_d);
    const double* prof[4];
    side_profiles(s, prof);
    fill_case(c, status_ptr(s), p.one, prof);
    p.one.upred = upred_ptr(s);
    Launch l;
    l.block = dim3(s->tx, s->ty, 1);
    l.grid = dim3((c.nx + s->tx - 1) / s->tx, (c.ny + s->ty - 1) / s->ty, 1);
    l.smem = s->smem;
    l.stream = s->stream;
    const StepFn step = kStep[c.precision][s->lat.q1 == 5][s->one_d];
    for (int k = 0; k < nsteps; ++k) {
        p.one.mac[0] = mac_ptr(s, s->cur);
        p.one.neq[0] = neq_ptr(s, s->cur);
        p.one.mac[1] = mac_ptr(s, 1 - s->cur);
        p.one.neq[1] = neq_ptr(s, 1 - s->cur);
        cudaError_t e = cudaSuccess;
        if (c.split == POND_SPLIT_INTERNAL) e = step(p, c.interp_order, true, l);   // predictor velocities
        if (e == cudaSuccess) e = step(p, c.interp_order, false, l);
        if (e != cudaSuccess) return cuda_status(e);
        if (c.split == POND_SPLIT_INTERNAL) {
            AuxParams a = aux_params(s, 1 - s->cur);   // new state; mac_prev = state before the step
            e = POND_BY_PRECISION(c.precision, internal_source, a, s->stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        s->cur = 1 - s->cur;
        s->steps += 1;
    }
    return POND_OK;
}

int pond_get_moments(pond_sim* s, double* rho, double* ux, double* uy, double* T, int on_device)
{
    if (!s) return POND_EINVAL;
    const long long N = (long long)s->cfg.nx * s->cfg.ny;
    AuxParams a = aux_params(s, s->cur);
    cudaError_t e;
    if (on_device) {
        e = POND_BY_PRECISION(s->cfg.precision, moments, a, rho, ux, uy, T, s->stream);
        if (e != cudaSuccess) return cuda_status(e);
    } else {
        const double* out[4] = {rho, ux, uy, T};
        const double* view[4];
        if (host_views(out, view)) {   // page-locked host memory: written in place
            e = POND_BY_PRECISION(s->cfg.precision, moments, a, const_cast<double*>(view[0]),
                                  const_cast<double*>(view[1]), const_cast<double*>(view[2]),
                                  const_cast<double*>(view[3]), s->stream);
            if (e != cudaSuccess) return cuda_status(e);
        } else {
            double* stage = mac_ptr(s, 1 - s->cur);
            e = POND_BY_PRECISION(s->cfg.precision, moments, a, stage, stage + N, stage + 2 * N, stage + 3 * N,
                                  s->stream);
            if (e != cudaSuccess) return cuda_status(e);
            double* dst[4] = {rho, ux, uy, T};
            for (int k = 0; k < 4; ++k) {
                if (!dst[k]) continue;
                e = cudaMemcpyAsync(dst[k], stage + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
                if (e != cudaSuccess) return cuda_status(e);
            }
        }
    }
    return sync_status(s);
}

int pond_get_populations(pond_sim* s, double* f, double* g, double* ux, double* uy, double* T, int on_device)
{
    if (!s) return POND_EINVAL;
    if (!on_device) return POND_EINVAL;
    AuxParams a = aux_params(s, s->cur);
    cudaError_t e = POND_BY_PRECISION(s->cfg.precision, get_pops, a, f, g, ux, uy, T, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return sync_status(s);
}

int pond_state_bytes(const pond_config* cfg, size_t* mac_bytes, size_t* neq_bytes)
{
    int rc = check_config(cfg);
    if (rc != POND_OK) return rc;
    if (!mac_bytes || !neq_bytes) return POND_EINVAL;
    const size_t N = (size_t)cfg->nx * (size_t)cfg->ny;
    *mac_bytes = NMAC * N * sizeof(double);
    *neq_bytes = (size_t)nneq(grad_order(*cfg)) * N * storage_bytes(cfg->precision);
    return POND_OK;
}

int pond_export_state(pond_sim* s, double* mac, void* neq, int on_device)
{
    if (!s || !mac || !neq) return POND_EINVAL;
    size_t mb = 0, nb = 0;
    pond_state_bytes(&s->cfg, &mb, &nb);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(mac, mac_ptr(s, s->cur), mb, kind, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(neq, neq_ptr(s, s->cur), nb, kind, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return sync_status(s);
}

int pond_import_state(pond_sim* s, const double* mac, const void* neq, int on_device)
{
    if (!s || !mac || !neq) return POND_EINVAL;
    size_t mb = 0, nb = 0;
    pond_state_bytes(&s->cfg, &mb, &nb);
    int rc = reset_status(s);
    if (rc != POND_OK) return rc;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(mac_ptr(s, s->cur), mac, mb, kind, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(neq_ptr(s, s->cur), neq, nb, kind, s->stream);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

int pond_get_stats(pond_sim* s, pond_stats* st)
{
    if (!s || !st) return POND_EINVAL;
    int rc = sync_status(s);
    if (rc == POND_ECUDA) return rc;
    const DevStatus& d = s->host_status;
    std::memset(st, 0, sizeof(*st));
    st->steps = s->steps;
    st->node_updates = s->steps * (long long)s->cfg.nx * s->cfg.ny;
    st->pc_iters_total = (int64_t)d.iters_total;
    st->pc_iters_max = (int32_t)d.iters_max;
    st->status = rc;
    st->nonconv_updates = (int64_t)d.nonconv;
    st->first_bad_node = d.first_bad == ~0ull ? -1 : (int64_t)d.first_bad;
    st->halo_fallbacks = (int64_t)d.fallbacks;
    return rc;
}

int pond_sync(pond_sim* s)
{
    if (!s) return POND_EINVAL;
    return sync_status(s);
}

int pond_destroy(pond_sim* s)
{
    if (!s) return POND_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    delete s;
    return cuda_status(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batched stepping
// ---------------------------------------------------------------------------------------
struct pond_batch {
    std::vector<pond_sim*> sims;
    cudaStream_t stream;
    CaseDesc* d_cases;
    int* d_tile_start;
    int* d_aux_start;
    std::vector<int> h_aux_start;  // host copy of d_aux_start
    int count, total_tiles, total_aux_blocks;
    bool any_internal;
    int flip;                      // parity of the steps taken since creation
    int graph_steps, graph_flip;
    cudaGraphExec_t graph;
    std::vector<cudaStream_t> member_streams;   // distinct member streams other than `stream`
    std::vector<cudaEvent_t> member_events;     // one per member stream
    cudaEvent_t done;                           // recorded on `stream` after each batch call
    std::vector<DevStatus> h_status_pageable;   // status read-back when no page-locked buffer
};

namespace {

size_t batch_layout(int32_t count, size_t* off_tiles, size_t* off_aux)
{
    size_t off = align_up((size_t)count * sizeof(CaseDesc));
    *off_tiles = off;
    off = align_up(off + (size_t)(count + 1) * sizeof(int));
    *off_aux = off;
    return align_up(off + (size_t)(count + 1) * sizeof(int));
}

cudaError_t batch_launch_step(pond_batch* b)
{
    pond_sim* s0 = b->sims[0];
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.lat = s0->lat;
    p.box_w = s0->box_w;
    p.box_h = s0->box_h;
    p.ahead = resident_step_blocks(s0->cfg, s0->one_d);
    p.flip = b->flip;
    p.ncase = b->count;
    p.cases = b->d_cases;
    p.tile_start = b->d_tile_start;
    Launch l;
    l.block = dim3(s0->tx, s0->ty, 1);
    l.grid = dim3(b->total_tiles, 1, 1);
    l.smem = s0->smem;
    l.stream = b->stream;
    const pond_config& c = s0->cfg;
    const StepFn step = kStep[c.precision][s0->lat.q1 == 5][s0->one_d];
    cudaError_t e = cudaSuccess;
    if (b->any_internal) e = step(p, c.interp_order, true, l);   // predictor velocities (internal split)
    if (e == cudaSuccess) e = step(p, c.interp_order, false, l);
    if (e == cudaSuccess && b->any_internal)
        e = POND_BY_PRECISION(c.precision, internal_source_batch, b->d_cases, b->d_aux_start, b->count,
                              b->flip, b->total_aux_blocks, b->stream);
    return e;
}

// Order the batch after work already queued on the members' streams, and the members'
// streams after the batch's work.
cudaError_t batch_wait_members(pond_batch* b)
{
    for (size_t k = 0; k < b->member_streams.size(); ++k) {
        cudaError_t e = cudaEventRecord(b->member_events[k], b->member_streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->member_events[k], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_release_members(pond_batch* b)
{
    if (b->member_streams.empty()) return cudaSuccess;
    cudaError_t e = cudaEventRecord(b->done, b->stream);
    for (size_t k = 0; k < b->member_streams.size() && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(b->member_streams[k], b->done, 0);
    return e;
}

void batch_destroy_events(pond_batch* b)
{
    for (cudaEvent_t ev : b->member_events) cudaEventDestroy(ev);
    b->member_events.clear();
    if (b->done) cudaEventDestroy(b->done);
    b->done = nullptr;
}

void batch_advance_members(pond_batch* b, int steps)
{
    for (pond_sim* s : b->sims) {
        if (steps % 2) s->cur = 1 - s->cur;
        s->steps += steps;
    }
}

}  // namespace

extern "C" int pond_batch_workspace_bytes(int32_t count, size_t* bytes)
{
    if (count < 1 || !bytes) return POND_EINVAL;
    size_t a, b;
    *bytes = batch_layout(count, &a, &b);
    return POND_OK;
}

extern "C" int pond_batch_create(pond_sim* const* sims, int32_t count, void* dev_workspace, size_t bytes,
                                 void* cuda_stream, pond_batch** out)
{
    if (!out) return POND_EINVAL;
    *out = nullptr;
    if (!sims || count < 1 || !dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign))
        return POND_EINVAL;
    size_t off_tiles, off_aux;
    if (bytes < batch_layout(count, &off_tiles, &off_aux)) return POND_ENOMEM;
    const pond_sim* s0 = sims[0];
    if (!s0) return POND_EINVAL;
    std::vector<CaseDesc> cases(count);
    std::vector<int> tile_start(count + 1), aux_start(count + 1);
    bool any_internal = false;
    int tiles = 0, aux = 0;
    for (int i = 0; i < count; ++i) {
        pond_sim* s = sims[i];
        if (!s) return POND_EINVAL;
        const pond_config& c = s->cfg;
        if (c.precision != s0->cfg.precision || c.lattice != s0->cfg.lattice ||
            c.interp_order != s0->cfg.interp_order || s->one_d != s0->one_d || s->tx != s0->tx ||
            s->ty != s0->ty || s->box_w != s0->box_w || s->box_h != s0->box_h)
            return POND_EINVAL;
        const double* prof[4];
        side_profiles(s, prof);
        fill_case(c, status_ptr(s), cases[i], prof);
        cases[i].upred = upred_ptr(s);
        cases[i].mac[0] = mac_ptr(s, s->cur);
        cases[i].neq[0] = neq_ptr(s, s->cur);
        cases[i].mac[1] = mac_ptr(s, 1 - s->cur);
        cases[i].neq[1] = neq_ptr(s, 1 - s->cur);
        cases[i].tiles_x = (c.nx + s->tx - 1) / s->tx;
        const long long t = (long long)cases[i].tiles_x * ((c.ny + s->ty - 1) / s->ty);
        const long long a = (cases[i].N + 255) / 256;
        if ((long long)tiles + t > (1ll << 30) || (long long)aux + a > (1ll << 30)) return POND_EINVAL;
        tile_start[i] = tiles;
        aux_start[i] = aux;
        tiles += (int)t;
        aux += (int)a;
        any_internal = any_internal || c.split == POND_SPLIT_INTERNAL;
    }
    tile_start[count] = tiles;
    aux_start[count] = aux;
    pond_batch* b = new (std::nothrow) pond_batch;
    if (!b) return POND_ENOMEM;
    b->sims.assign(sims, sims + count);
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    char* ws = reinterpret_cast<char*>(dev_workspace);
    b->d_cases = reinterpret_cast<CaseDesc*>(ws);
    b->d_tile_start = reinterpret_cast<int*>(ws + off_tiles);
    b->d_aux_start = reinterpret_cast<int*>(ws + off_aux);
    b->count = count;
    b->total_tiles = tiles;
    b->total_aux_blocks = aux;
    b->h_aux_start = aux_start;
    b->any_internal = any_internal;
    b->flip = 0;
    b->graph_steps = 0;
    b->graph_flip = 0;
    b->graph = nullptr;
    b->done = nullptr;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < count; ++i) {
        cudaStream_t ms = sims[i]->stream;
        bool seen = (ms == b->stream);
        for (cudaStream_t t : b->member_streams) seen = seen || (t == ms);
        if (!seen) b->member_streams.push_back(ms);
    }
    for (size_t k = 0; k < b->member_streams.size() && e == cudaSuccess; ++k) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->member_events.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = batch_wait_members(b);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_cases, cases.data(), count * sizeof(CaseDesc),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tile_start, tile_start.data(), (count + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_aux_start, aux_start.data(), (count + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        batch_destroy_events(b);
        delete b;
        return cuda_status(e);
    }
    *out = b;
    return POND_OK;
}

extern "C" int pond_batch_use_graph(pond_batch* b, int32_t steps_per_graph)
{
    if (!b || steps_per_graph < 0 || steps_per_graph % 2) return POND_EINVAL;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = 0;
    if (steps_per_graph == 0) return POND_OK;
    if (!b->stream) return POND_EINVAL;   // the legacy default stream cannot be captured
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    const int flip0 = b->flip;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < steps_per_graph && le == cudaSuccess; ++k) {
        le = batch_launch_step(b);
        b->flip ^= 1;
    }
    b->flip = flip0;
    e = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(le != cudaSuccess ? le : e);
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_status(e);
    }
    b->graph_steps = steps_per_graph;
    b->graph_flip = flip0;
    return POND_OK;
}

extern "C" int pond_batch_step(pond_batch* b, int32_t nsteps)
{
    if (!b || nsteps < 0) return POND_EINVAL;
    cudaError_t we = batch_wait_members(b);
    if (we != cudaSuccess) return cuda_status(we);
    int left = nsteps;
    while (left > 0) {
        if (b->graph && left >= b->graph_steps && b->flip == b->graph_flip) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return cuda_status(e);
            batch_advance_members(b, b->graph_steps);   // even: the parity is unchanged
            left -= b->graph_steps;
            continue;
        }
        cudaError_t e = batch_launch_step(b);
        if (e != cudaSuccess) return cuda_status(e);
        b->flip ^= 1;
        batch_advance_members(b, 1);
        --left;
    }
    return cuda_status(batch_release_members(b));
}

extern "C" int pond_batch_destroy(pond_batch* b)
{
    if (!b) return POND_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    batch_destroy_events(b);
    delete b;
    return cuda_status(e);
}

namespace {

// Read every member's status block into its handle with one synchronisation of the batch's
// stream; returns the worst sticky status (non-physical before non-convergence).
// Page-locked status blocks for the batch read-backs of this host thread, grown to the
// largest batch seen and kept (allocating or freeing page-locked memory synchronises the
// device, so a batch that is rebuilt often must not do it); null if the allocation fails.
DevStatus* pinned_status_array(int count)
{
    static thread_local DevStatus* buf = nullptr;
    static thread_local int cap = 0;
    if (count <= cap) return buf;
    void* p = nullptr;
    if (cudaMallocHost(&p, (size_t)count * sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (buf) cudaFreeHost(buf);
    buf = static_cast<DevStatus*>(p);
    cap = count;
    return buf;
}

int batch_read_status(pond_batch* b, bool* input_bad)
{
    DevStatus* h = pinned_status_array(b->count);
    if (!h) {
        b->h_status_pageable.resize(b->count);
        h = b->h_status_pageable.data();
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(h + i, status_ptr(b->sims[i]), sizeof(DevStatus), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = POND_OK;
    if (input_bad) *input_bad = false;
    for (int i = 0; i < b->count; ++i) {
        b->sims[i]->host_status = h[i];
        if (input_bad && (h[i].flags & kInputBad)) *input_bad = true;
        if (h[i].flags & 1) rc = POND_ENONPHYSICAL;
        else if ((h[i].flags & 2) && rc == POND_OK) rc = POND_ENOCONV;
    }
    return rc;
}

}  // namespace

// Runs launch(c0, c1, block0, blocks, fields) over the batch's members in chunks of kAuxChunk;
// fields.f[c - c0][k] = field(c, k).  One launch per chunk: the aux blocks of members [c0, c1)
// are block0 .. block0 + blocks - 1 of the batch's aux block numbering.
template <class F, class L>
cudaError_t for_member_chunks(const pond_batch* b, F field, L launch)
{
    for (int c0 = 0; c0 < b->count; c0 += kAuxChunk) {
        const int c1 = std::min(b->count, c0 + kAuxChunk);
        MemberFields fld;
        std::memset(&fld, 0, sizeof(fld));
        for (int c = c0; c < c1; ++c)
            for (int k = 0; k < 4; ++k) fld.f[c - c0][k] = field(c, k);
        const int block0 = b->h_aux_start[c0];
        cudaError_t e = launch(c0, c1, block0, b->h_aux_start[c1] - block0, fld);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" int pond_batch_set_state(pond_batch* b, const double* const* rho, const double* const* ux,
                                    const double* const* uy, const double* const* T, int on_device)
{
    if (!b || !rho || !ux || !uy || !T) return POND_EINVAL;
    for (int i = 0; i < b->count; ++i)
        if (!rho[i] || !ux[i] || !uy[i] || !T[i]) return POND_EINVAL;
    cudaError_t e = batch_wait_members(b);
    if (e != cudaSuccess) return cuda_status(e);
    const double* const* in[4] = {rho, ux, uy, T};
    for (pond_sim* s : b->sims) s->steps = 0;
    // every member's status block cleared by one launch, the input checked and the equilibria
    // set by one launch per kAuxChunk members
    reset_status_batch_kernel<<<(unsigned int)((b->count + 127) / 128), 128, 0, b->stream>>>(b->d_cases, b->count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
    auto staged = [b](int c, int k) {        // host input: staged in the member's idle buffer
        pond_sim* s = b->sims[c];
        return mac_ptr(s, 1 - s->cur) + k * (long long)s->cfg.nx * s->cfg.ny;
    };
    if (!on_device) {
        // page-locked input: read in place by the staging kernel; other host memory: copied
        std::vector<double*> view(4 * (size_t)b->count, nullptr);
        bool page_locked = true;
        for (int i = 0; i < b->count && page_locked; ++i) {
            const double* src[4] = {in[0][i], in[1][i], in[2][i], in[3][i]};
            const double* v[4];
            page_locked = host_views(src, v);
            for (int k = 0; k < 4; ++k) view[4 * (size_t)i + k] = const_cast<double*>(v[k]);
        }
        if (page_locked) {
            e = for_member_chunks(
                b, [&](int c, int k) { return view[4 * (size_t)c + k]; },
                [b](int c0, int c1, int block0, int blocks, const MemberFields& fld) {
                    stage_check_batch_kernel<<<blocks, 256, 0, b->stream>>>(b->d_cases, b->d_aux_start, c0, c1,
                                                                            block0, b->flip, fld);
                    return cudaGetLastError();
                });
        } else {
            for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
                pond_sim* s = b->sims[i];
                const long long N = (long long)s->cfg.nx * s->cfg.ny;
                for (int k = 0; k < 4 && e == cudaSuccess; ++k)
                    e = cudaMemcpyAsync(staged(i, k), in[k][i], N * sizeof(double), cudaMemcpyHostToDevice,
                                        b->stream);
            }
            if (e == cudaSuccess)
                e = for_member_chunks(b, staged, [b](int c0, int c1, int block0, int blocks, const MemberFields& fld) {
                    check_fields_batch_kernel<<<blocks, 256, 0, b->stream>>>(b->d_cases, b->d_aux_start, c0, c1,
                                                                             block0, fld);
                    return cudaGetLastError();
                });
        }
        if (e != cudaSuccess) return cuda_status(e);
        // one synchronisation for every member's check
        bool bad = false;
        const int rc = batch_read_status(b, &bad);
        if (rc == POND_ECUDA) return rc;
        if (bad) {
            for (int i = 0; i < b->count; ++i) {
                const int r = reset_status(b->sims[i]);
                if (r != POND_OK) return r;
            }
            return POND_EINVAL;
        }
    }
    const int precision = b->sims[0]->cfg.precision;
    e = for_member_chunks(
        b,
        [&](int c, int k) { return on_device ? const_cast<double*>(in[k][c]) : staged(c, k); },
        [b, precision](int c0, int c1, int block0, int blocks, const MemberFields& fld) {
            return POND_BY_PRECISION(precision, init_batch, b->d_cases, b->d_aux_start, c0, c1, block0, blocks,
                                     b->flip, fld, b->stream);
        });
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(batch_release_members(b));
}

extern "C" int pond_batch_get_moments(pond_batch* b, double* const* rho, double* const* ux, double* const* uy,
                                      double* const* T, int on_device)
{
    if (!b) return POND_EINVAL;
    cudaError_t e = batch_wait_members(b);
    if (e != cudaSuccess) return cuda_status(e);
    double* const* out[4] = {rho, ux, uy, T};
    // device or page-locked host outputs: written in place by one launch per kAuxChunk members
    std::vector<double*> direct(4 * (size_t)b->count, nullptr);
    bool all_direct = true;
    for (int i = 0; i < b->count && all_direct; ++i) {
        const double* dst[4];
        for (int k = 0; k < 4; ++k) dst[k] = out[k] ? out[k][i] : nullptr;
        const double* view[4];
        if (on_device) {
            for (int k = 0; k < 4; ++k) view[k] = dst[k];
        } else {
            all_direct = host_views(dst, view);
        }
        for (int k = 0; k < 4; ++k) direct[4 * (size_t)i + k] = const_cast<double*>(view[k]);
    }
    if (all_direct) {
        const int precision = b->sims[0]->cfg.precision;
        e = for_member_chunks(
            b, [&](int c, int k) { return direct[4 * (size_t)c + k]; },
            [b, precision](int c0, int c1, int block0, int blocks, const MemberFields& fld) {
                return POND_BY_PRECISION(precision, moments_batch, b->d_cases, b->d_aux_start, c0, c1, block0,
                                         blocks, b->flip, fld, b->stream);
            });
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int i = 0; i < b->count && !all_direct; ++i) {   // pageable host memory: staged copies
        pond_sim* s = b->sims[i];
        const long long N = (long long)s->cfg.nx * s->cfg.ny;
        double* dst[4] = {rho ? rho[i] : nullptr, ux ? ux[i] : nullptr, uy ? uy[i] : nullptr, T ? T[i] : nullptr};
        AuxParams a = aux_params(s, s->cur);
        const double* cdst[4] = {dst[0], dst[1], dst[2], dst[3]};
        const double* view[4];
        if (host_views(cdst, view)) {   // page-locked host memory: written in place
            e = POND_BY_PRECISION(s->cfg.precision, moments, a, const_cast<double*>(view[0]),
                                  const_cast<double*>(view[1]), const_cast<double*>(view[2]),
                                  const_cast<double*>(view[3]), b->stream);
        } else {
            double* stage = mac_ptr(s, 1 - s->cur);
            e = POND_BY_PRECISION(s->cfg.precision, moments, a, stage, stage + N, stage + 2 * N, stage + 3 * N,
                                  b->stream);
            for (int k = 0; k < 4 && e == cudaSuccess; ++k)
                if (dst[k])
                    e = cudaMemcpyAsync(dst[k], stage + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    const int rc = batch_read_status(b, nullptr);
    if (rc == POND_ECUDA) return rc;
    e = batch_release_members(b);
    return e != cudaSuccess ? cuda_status(e) : rc;
}

// ---------------------------------------------------------------------------------------
// Launch-shape autotuning
// ---------------------------------------------------------------------------------------
namespace {

// Problem class of a tuning result: everything that selects the kernel, the boundary
// handling and the grid size rounded up to powers of two.
struct TuneKey {
    int precision, lattice, order, split, one_d, bc_x, bc_y, lx, ly;
    bool operator<(const TuneKey& o) const
    {
        const int a[9] = {precision, lattice, order, split, one_d, bc_x, bc_y, lx, ly};
        const int b[9] = {o.precision, o.lattice, o.order, o.split, o.one_d, o.bc_x, o.bc_y, o.lx, o.ly};
        for (int k = 0; k < 9; ++k)
            if (a[k] != b[k]) return a[k] < b[k];
        return false;
    }
};

int ceil_log2(int v)
{
    int k = 0;
    while ((1 << k) < v && k < 30) ++k;
    return k;
}

TuneKey tune_key(const pond_config& c)
{
    return TuneKey{c.precision, c.lattice, c.interp_order, c.split, c.ny == 1, c.bc_x, c.bc_y,
                   ceil_log2(c.nx), ceil_log2(c.ny)};
}

std::mutex g_tune_mutex;
std::map<TuneKey, pond_tuning> g_tune_cache;

// Time `steps` steps (after one warm-up step) of a copy of s's current state under one launch
// shape, on s's stream, in the scratch workspace.  Returns POND_OK and the time per step, or
// the status that ruled the shape out.
int time_shape(pond_sim* s, void* scratch, size_t bytes, int tile_x, int tile_y, int halo, int steps,
               cudaEvent_t e0, cudaEvent_t e1, double* ms)
{
    pond_config c = s->cfg;
    c.tile_x = tile_x;
    c.tile_y = tile_y;
    c.halo = halo;
    pond_sim* t = nullptr;
    int rc = pond_create(&c, scratch, bytes, s->stream, &t);
    if (rc != POND_OK) return rc;
    size_t mb = 0, nb = 0;
    pond_state_bytes(&s->cfg, &mb, &nb);
    cudaError_t e = cudaMemcpyAsync(mac_ptr(t, t->cur), mac_ptr(s, s->cur), mb, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(neq_ptr(t, t->cur), neq_ptr(s, s->cur), nb, cudaMemcpyDeviceToDevice, s->stream);
    for (int w = 0; w < 4 && e == cudaSuccess; ++w)   // and the prescribed sides' profiles
        if (s->lay.prof[w])
            e = cudaMemcpyAsync(prof_ptr(t, w), prof_ptr(s, w), 4 * (size_t)side_length(c, w) * sizeof(double),
                                cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) {
        pond_destroy(t);
        return cuda_status(e);
    }
    rc = pond_step(t, 1);
    if (rc == POND_OK) rc = cuda_status(cudaEventRecord(e0, s->stream));
    if (rc == POND_OK) rc = pond_step(t, steps);
    if (rc == POND_OK) rc = cuda_status(cudaEventRecord(e1, s->stream));
    if (rc == POND_OK) {
        // kernel-side outcomes of the copy (a node that hit the iteration cap, a non-physical
        // node) do not change the work timed; only runtime failures rule the shape out
        rc = sync_status(t);
        if (rc == POND_ENOCONV || rc == POND_ENONPHYSICAL) rc = POND_OK;
    }
    float f = 0.f;
    if (rc == POND_OK) rc = cuda_status(cudaEventElapsedTime(&f, e0, e1));
    const int rd = pond_destroy(t);
    if (rc == POND_OK) rc = rd;
    *ms = (double)f / steps;
    return rc;
}

}  // namespace

extern "C" int pond_get_launch(pond_sim* s, pond_tuning* out)
{
    if (!s || !out) return POND_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->tile_x = s->tx;
    out->tile_y = s->ty;
    out->halo = s->cfg.halo;
    return POND_OK;
}

extern "C" int pond_set_launch(pond_sim* s, int32_t tile_x, int32_t tile_y, int32_t halo)
{
    if (!s) return POND_EINVAL;
    return apply_shape(s, tile_x, tile_y, halo);
}

extern "C" int pond_autotune(pond_sim* s, void* dev_scratch, size_t bytes, int32_t steps, int32_t flags,
                             pond_tuning* out)
{
    if (!s || !out || steps < 1 || steps > 1000 || (flags & ~(POND_TUNE_APPLY | POND_TUNE_RETIME)))
        return POND_EINVAL;
    std::memset(out, 0, sizeof(*out));
    const TuneKey key = tune_key(s->cfg);
    if (!(flags & POND_TUNE_RETIME)) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *out = it->second;
            out->candidates = 0;
            return (flags & POND_TUNE_APPLY) ? apply_shape(s, out->tile_x, out->tile_y, out->halo) : POND_OK;
        }
    }
    if (!dev_scratch || (reinterpret_cast<uintptr_t>(dev_scratch) % kAlign)) return POND_EINVAL;
    if (bytes < layout_of(s->cfg).total) return POND_ENOMEM;
    // candidates: every 2-D tile of 256 nodes with an even width from 8 x 32 to 128 x 2, and
    // box halos that cover the footprint of cool (4) to hot (8) gas
    static const int tiles2d[5][2] = {{32, 8}, {16, 16}, {64, 4}, {128, 2}, {8, 32}};
    static const int halos[4] = {4, 5, 6, 8};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = cuda_status(e);
    struct Trial { double ms; int tx, ty, halo; };
    std::vector<Trial> trials;
    const int ntiles = s->one_d ? 1 : 5;
    for (int ti = 0; ti < ntiles && rc == POND_OK; ++ti) {
        const int tx = s->one_d ? 0 : tiles2d[ti][0], ty = s->one_d ? 0 : tiles2d[ti][1];
        for (int hi = 0; hi < 4 && rc == POND_OK; ++hi) {
            double ms = 0.0;
            const int r = time_shape(s, dev_scratch, bytes, tx, ty, halos[hi], steps, e0, e1, &ms);
            if (r == POND_ECUDA) rc = r;           // a runtime failure ends the search
            if (r != POND_OK) continue;            // shape ruled out (shared memory, state)
            trials.push_back(Trial{ms, tx, ty, halos[hi]});
        }
    }
    // the candidates lie within a few per cent of each other: time the three fastest twice
    // more and keep each one's best, so that one noisy trial does not decide
    std::sort(trials.begin(), trials.end(), [](const Trial& a, const Trial& b) { return a.ms < b.ms; });
    const size_t finalists = std::min<size_t>(3, trials.size());
    for (int rep = 0; rep < 2 && rc == POND_OK && finalists > 1; ++rep)
        for (size_t k = 0; k < finalists && rc == POND_OK; ++k) {
            double ms = 0.0;
            const int r = time_shape(s, dev_scratch, bytes, trials[k].tx, trials[k].ty, trials[k].halo, steps,
                                     e0, e1, &ms);
            if (r == POND_ECUDA) rc = r;
            if (r == POND_OK) trials[k].ms = std::min(trials[k].ms, ms);
        }
    std::sort(trials.begin(), trials.begin() + finalists,
              [](const Trial& a, const Trial& b) { return a.ms < b.ms; });
    const int tried = (int)trials.size();
    const double best = tried ? trials[0].ms : 0.0;
    const int bx = tried ? (s->one_d ? kStepThreads1D : trials[0].tx) : 0;
    const int by = tried ? (s->one_d ? 1 : trials[0].ty) : 0;
    const int bh = tried ? trials[0].halo : 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != POND_OK) return rc;
    if (tried == 0) return POND_EINVAL;
    out->tile_x = bx;
    out->tile_y = by;
    out->halo = bh;
    out->candidates = tried;
    out->ms_per_step = best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = *out;
    }
    return (flags & POND_TUNE_APPLY) ? apply_shape(s, s->one_d ? 0 : bx, s->one_d ? 0 : by, bh) : POND_OK;
}

extern "C" void pond_autotune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.clear();
}

// ---------------------------------------------------------------------------------------
// Allocation-free stepping (pond_step_static): the second copy of the state and the status
// block live in this file-scope device array instead of a caller workspace.
// ---------------------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_pond_static_scratch[POND_STATIC_SCRATCH_BYTES];

constexpr int kStaticMaxDevices = 64;

// Driver calls that identify the current context (resolved once through the runtime, so the
// library does not link the driver library itself).  A context's ID is never reused within a
// process, so a changed ID means the context was reset or replaced.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
std::once_flag g_ctx_fns_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// ID of the context current on this thread; 0 if none is current yet.
int current_context_id(unsigned long long* id)
{
    std::call_once(g_ctx_fns_once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return POND_ECUDA;
    void* ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0) return POND_ECUDA;
    *id = 0;
    if (ctx && g_ctx_get_id(ctx, id) != 0) return POND_ECUDA;
    return POND_OK;
}

// Per-device set-up of the allocation-free path, valid for one context: the array's device
// address (its name in host code is only a stand-in), the SM count, and the launch shapes
// already prepared (preparing one sets the step kernel's shared-memory limit).
struct StaticShape {
    int precision, lattice, interp_order, tile_x, tile_y, halo, one_d;
    Shape sh;
};
struct StaticDevice {
    unsigned long long ctx = 0;
    void* addr = nullptr;
    int sms = 0;
    std::vector<StaticShape> shapes;
};
std::mutex g_static_mutex;
StaticDevice g_static[kStaticMaxDevices];

// The device's set-up for the current context (device dev current), done on first use and
// again whenever the current context has changed.
int static_device(int dev, StaticDevice** out)
{
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticDevice& d = g_static[dev];
    unsigned long long ctx = 0;
    int rc = current_context_id(&ctx);
    if (rc != POND_OK) return rc;
    if (!d.addr || ctx == 0 || ctx != d.ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pond_static_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_status(e);
        rc = current_context_id(&ctx);       // the look-up made the device's context current
        if (rc != POND_OK) return rc;
        d.ctx = ctx;
        d.addr = p;
        d.sms = sms;
        d.shapes.clear();
    }
    *out = &d;
    return POND_OK;
}

// The launch shape for cfg on device d, prepared on first use (make_shape sets the kernel's
// shared-memory limit) and reused afterwards.
int static_shape(StaticDevice* d, const pond_config& c, Shape* out)
{
    std::lock_guard<std::mutex> lock(g_static_mutex);
    const int one_d = c.ny == 1;
    for (const StaticShape& s : d->shapes)
        if (s.precision == c.precision && s.lattice == c.lattice && s.interp_order == c.interp_order &&
            s.tile_x == c.tile_x && s.tile_y == c.tile_y && s.halo == c.halo && s.one_d == one_d) {
            *out = s.sh;
            return POND_OK;
        }
    StaticShape s{c.precision, c.lattice, c.interp_order, c.tile_x, c.tile_y, c.halo, one_d, Shape()};
    int rc = make_shape(c, c.tile_x, c.tile_y, c.halo, &s.sh);
    if (rc != POND_OK) return rc;
    d->shapes.push_back(s);
    *out = s.sh;
    return POND_OK;
}

}  // namespace

extern "C" int pond_step_static(const pond_config* cfg, double* mac, void* neq, int32_t nsteps,
                                void* cuda_stream, pond_stats* stats)
{
    int rc = check_config(cfg);
    if (rc != POND_OK) return rc;
    if (!mac || !neq || nsteps < 0) return POND_EINVAL;
    size_t mb = 0, nb = 0;
    pond_state_bytes(cfg, &mb, &nb);
    const size_t off_neq = align_up(mb), off_status = off_neq + align_up(nb);
    // internal split: the predictor velocities follow the status block
    const size_t off_upred = off_status + align_up(sizeof(DevStatus));
    const size_t need = off_upred + (cfg->split == POND_SPLIT_INTERNAL ? align_up(upred_bytes(*cfg)) : 0);
    if (need > (size_t)POND_STATIC_SCRATCH_BYTES) return POND_ENOMEM;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kStaticMaxDevices) return POND_EINVAL;
    StaticDevice* sd = nullptr;
    rc = static_device(dev, &sd);
    if (rc != POND_OK) return rc;
    char* scratch = reinterpret_cast<char*>(sd->addr);
    double* smac = reinterpret_cast<double*>(scratch);
    void* sneq = scratch + off_neq;
    DevStatus* st = reinterpret_cast<DevStatus*>(scratch + off_status);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);

    // launch shape of the step kernel, as pond_create chooses it
    Shape sh;
    rc = static_shape(sd, *cfg, &sh);
    if (rc != POND_OK) return rc;
    const bool one_d = sh.one_d;
    const int tx = sh.tx, ty = sh.ty, box_w = sh.box_w, box_h = sh.box_h;
    const size_t smem = sh.smem;
    const Lattice lat = make_lattice(cfg->lattice == POND_D2Q16 ? 4 : 5);

    // the array keeps the previous call's contents: clear the status block
    e = cudaMemsetAsync(st, 0, sizeof(DevStatus), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st->first_bad, 0xff, sizeof(st->first_bad), stream);
    if (e != cudaSuccess) return cuda_status(e);

    const long long N = (long long)cfg->nx * cfg->ny;
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.lat = lat;
    p.box_w = box_w;
    p.box_h = box_h;
    // the next-wave L2 prefetch distance, as pond_step sets it: the blocks resident at once
    p.ahead = sd->sms * step_blocks_per_sm(one_d, cfg->lattice == POND_D2Q25, cfg->precision == POND_FP64);
    fill_case(*cfg, st, p.one);
    p.one.upred = cfg->split == POND_SPLIT_INTERNAL ? reinterpret_cast<double*>(scratch + off_upred) : nullptr;
    Launch l;
    l.block = dim3(tx, ty, 1);
    l.grid = dim3((cfg->nx + tx - 1) / tx, (cfg->ny + ty - 1) / ty, 1);
    l.smem = smem;
    l.stream = stream;
    AuxParams a;
    std::memset(&a, 0, sizeof(a));
    a.lat = lat;
    a.nx = cfg->nx;
    a.ny = cfg->ny;
    a.bc_x = cfg->bc_x;
    a.bc_y = cfg->bc_y;
    a.split = cfg->split;
    a.nord = grad_order(*cfg);
    std::memcpy(a.wall, cfg->wall, sizeof(a.wall));
    a.N = N;
    a.cv = p.one.cv;
    a.mu = cfg->mu;
    a.status = st;
    // ping-pong between the caller's buffers and the array
    for (int k = 0; k < nsteps; ++k) {
        const bool from_caller = (k % 2 == 0);
        p.one.mac[0] = from_caller ? mac : smac;
        p.one.neq[0] = from_caller ? neq : sneq;
        p.one.mac[1] = from_caller ? smac : mac;
        p.one.neq[1] = from_caller ? sneq : neq;
        const StepFn step = kStep[cfg->precision][lat.q1 == 5][one_d];
        e = cudaSuccess;
        if (cfg->split == POND_SPLIT_INTERNAL) e = step(p, cfg->interp_order, true, l);   // predictor
        if (e == cudaSuccess) e = step(p, cfg->interp_order, false, l);
        if (e != cudaSuccess) return cuda_status(e);
        if (cfg->split == POND_SPLIT_INTERNAL) {
            a.mac = p.one.mac[1];
            a.neq = p.one.neq[1];
            a.mac_prev = p.one.mac[0];
            e = POND_BY_PRECISION(cfg->precision, internal_source, a, stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    if (nsteps % 2 == 1) {   // the last step wrote into the array: copy the result back
        e = cudaMemcpyAsync(mac, smac, mb, cudaMemcpyDeviceToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(neq, sneq, nb, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (!stats) return POND_OK;
    DevStatus h;
    e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    std::memset(stats, 0, sizeof(*stats));
    stats->steps = nsteps;
    stats->node_updates = (int64_t)nsteps * N;
    stats->pc_iters_total = (int64_t)h.iters_total;
    stats->pc_iters_max = (int32_t)h.iters_max;
    stats->nonconv_updates = (int64_t)h.nonconv;
    stats->first_bad_node = h.first_bad == ~0ull ? -1 : (int64_t)h.first_bad;
    stats->halo_fallbacks = (int64_t)h.fallbacks;
    stats->status = (h.flags & 1) ? POND_ENONPHYSICAL : (h.flags & 2) ? POND_ENOCONV : POND_OK;
    return stats->status;
}
