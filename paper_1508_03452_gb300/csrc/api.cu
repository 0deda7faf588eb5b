// api.cu -- host implementation of the lbrmhd C ABI (include/lbrmhd.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "aux.cuh"
#include "lbrmhd.h"

namespace {

thread_local std::string g_create_error;

struct RunState {
    lbrmhd_params p{};
    int64_t N = 0, stride = 0;
    void* pops[2] = {nullptr, nullptr};  // f, g: 9 group planes of 4-vectors, then the rest pairs (fg_elem)
    void* h[2] = {nullptr, nullptr};     // h: 12 pair planes of 2-vectors, then h_24 (h_elem)
    void* prim[2] = {nullptr, nullptr};  // 3 planes of primitive 4-vectors (prim_elem)
    int cur = 0;
    bool initialized = false;
    lb::RefState ref{1.0, 4.0, 1.0};
    double means[lb::NMEANS] = {};               // reference-state means (see means_kernel)
    double Er[3] = {0, 0, 0}, Br[3] = {0, 0, 0};  // reference fields of the h deviations
    double Xr[3][3] = {}, Yr[3] = {};            // reference EM terms of the f deviations
    lb::RefPops refpops{};
    lb::HalfScale hs{};
    unsigned long long* d_stats = nullptr;  // lb::kStatSlots x lb::kNumStats recovery counters
    int64_t steps = 0;
    int periodic[3] = {1, 1, 1};
    float* d_samples = nullptr;  // caller-owned training-sample buffer (or NULL)
    void* d_ez0 = nullptr;       // E^z of the initial state (primitive type, N), for the reconnection rate
    double* d_drive = nullptr;   // drive velocity (driven runs) or body force (forced runs) per (x, y) column
    double* d_umax = nullptr;    // forced runs with a cut-off: max |u|^2 of the state, running max of the next
    // tensor maps of the TMA tile kernel for input buffer 0 and 1 (empty: the run takes the per-cell kernel)
    std::vector<lb::TileMaps> tmaps;
    int4* d_edge = nullptr;  // the run's edge tiles (32 x 4 cells) for the per-cell launch beside the tile kernel
    int nedge = 0;
};

constexpr size_t kStatsBytes = lb::kNumStats * sizeof(unsigned long long);  // totals (checkpoint)
constexpr size_t kStatsAlloc = (size_t)lb::kStatSlots * kStatsBytes;       // per-slot copies on the device

size_t pop_bytes(int precision) { return precision == LBRMHD_FP64 ? 8 : (precision == LBRMHD_FP32 ? 4 : 2); }
size_t hp_bytes(int precision) { return precision == LBRMHD_FP64 ? 8 : 4; }

}  // namespace

struct lbrmhd_state_s {
    std::vector<RunState> runs;
    int precision = LBRMHD_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    double* d_scratch = nullptr;  // per-block partial sums (diagnostics, reference means)
    int64_t scratch_blocks = 0;
    double* d_io = nullptr;  // staging for inputs / outputs
    size_t io_bytes = 0;
    double* d_small = nullptr;  // 32 float64
    int* d_flag = nullptr;
    double* d_noalloc = nullptr;  // device address of g_noalloc_partials in this handle's context
    int* d_status = nullptr;      // lb::STATUS_* bits raised by the step kernels
    int sms = 1;                  // multiprocessors of the device
    unsigned int* d_barrier = nullptr;  // arrival counter of the persistent launch's grid barrier
    unsigned char* d_mlp = nullptr;  // packed network of the learned seed
    bool mlp_set = false;
    // launch schedule (lbrmhd_set_schedule / lbrmhd_autotune)
    lbrmhd_schedule sched{LBRMHD_SCHED_PER_RUN, 128, 0, 0, 1, 0};
    // streams of the multi-stream per-run schedule, with their fork / join events
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_join;
    cudaEvent_t ev_fork = nullptr;
    // batched launches: per-run arguments for both input buffers, tile list
    void* d_args = nullptr;       // 2 x runs StepArgs<Cfg> records (input buffer 0, then 1), 16-byte stride
    bool args_dirty = true;
    int4* d_tiles = nullptr;
    size_t tiles_cap = 0;
    struct Group {
        bool is3d, open;
        int seed, first, count;
    };
    std::vector<Group> groups;
    bool tiles_dirty = true;
    // CUDA graphs of graph_steps steps, one per starting input buffer
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_len = 0;
};

#define LB_CK(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return LBRMHD_ERR_CUDA;                                                        \
        }                                                                                  \
    } while (0)

namespace {

int fail(lbrmhd_handle h, int code, const std::string& msg)
{
    h->err = msg;
    return code;
}

bool bad_run(lbrmhd_handle h, int run) { return !h || run < 0 || run >= (int)h->runs.size(); }

struct RunRef {
    const double *Er, *Br;
    const double (*Xr)[3];
    const double* Yr;
};

template <class R>
lb::Phys<R> make_phys(const lbrmhd_params& p, const lb::RefState& ref, const RunRef& rr)
{
    const double* Er = rr.Er;
    const double* Br = rr.Br;
    lb::Phys<R> k{};
    const double dt = p.dx / (std::sqrt(2.0) * p.c);
    const double C = lb::kQ * p.c * dt / p.dx;
    k.c = (R)p.c;
    k.c2 = (R)(p.c * p.c);
    k.inv_c = (R)(1.0 / p.c);
    k.eps0 = (R)(1.0 / (p.c * p.c));
    k.sigma = (R)p.sigma;
    k.inv_tau = (R)(1.0 / p.tau);
    k.half_dt_c2 = (R)(0.5 * dt * p.c * p.c);
    k.inv_half_dt_c2 = (R)(1.0 / (0.5 * dt * p.c * p.c));
    k.gm1 = (R)(p.gamma_ad - 1.0);
    k.C = (R)C;
    // LBRMHD_FLAG_FIRST_ORDER_FLUX: the limiter's correction term off, i.e. plain first-order upwind
    k.kappa = (p.flags & LBRMHD_FLAG_FIRST_ORDER_FLUX) ? (R)0 : (R)(0.5 * (1.0 - C));
    k.kvisc = (R)(p.alpha * p.c * dt / p.dx);
    k.n_r = (R)ref.n_r;
    k.eps_r = (R)ref.eps_r;
    k.p_r = (R)ref.p_r;
    k.dx = (R)p.dx;
    const double eps0 = 1.0 / (p.c * p.c);
    for (int a = 0; a < 3; ++a) {
        k.Er[a] = (R)Er[a];
        k.Br[a] = (R)Br[a];
        for (int b = 0; b < 3; ++b)
            k.dXr[a][b] = (R)(rr.Xr[a][b] - eps0 * (Er[a] * Er[b] + p.c * p.c * Br[a] * Br[b]));
    }
    const double BxE[3] = {Br[1] * Er[2] - Br[2] * Er[1], Br[2] * Er[0] - Br[0] * Er[2], Br[0] * Er[1] - Br[1] * Er[0]};
    for (int a = 0; a < 3; ++a) k.dYr[a] = (R)(rr.Yr[a] - eps0 * p.c * BxE[a]);
    // moments of the reference EM terms: T^00 = tr X / 2, T^0a = -Y_a, T^ab = -X_ab + tr X / 2 d_ab
    const double tr = rr.Xr[0][0] + rr.Xr[1][1] + rr.Xr[2][2];
    k.Tem[0] = (R)(0.5 * tr);
    for (int a = 0; a < 3; ++a) k.Tem[1 + a] = (R)(-rr.Yr[a]);
    for (int a = 0; a < 3; ++a) k.Tem[4 + a] = (R)(-rr.Xr[a][a] + 0.5 * tr);
    k.Tem[7] = (R)(-rr.Xr[0][1]);
    k.Tem[8] = (R)(-rr.Xr[0][2]);
    k.Tem[9] = (R)(-rr.Xr[1][2]);
    const bool f64 = p.precision == LBRMHD_FP64;
    k.tol = (R)(p.tol > 0 ? p.tol : (f64 ? 1e-14 : 1e-6));
    k.maxit = p.max_iters > 0 ? p.max_iters : 64;
    return k;
}

RunRef runref(const RunState& r) { return RunRef{r.Er, r.Br, r.Xr, r.Yr}; }

template <class Cfg>
lb::PopView<Cfg> view(const RunState& r, int buf)
{
    lb::PopView<Cfg> v{};
    v.fg = (typename Cfg::pop*)r.pops[buf];
    v.h = (typename Cfg::hpop*)r.h[buf];
    v.prim = (typename Cfg::prim*)r.prim[buf];
    v.nx = r.p.nx;
    v.ny = r.p.ny;
    v.nz = r.p.nz;
    v.stride = r.stride;
    for (int a = 0; a < 3; ++a) v.periodic[a] = r.periodic[a];
    v.hs = r.hs;
    return v;
}

// reference state of the deviations, from the means of the initial fields
// (means_kernel layout): the rest equilibrium of (n_r, p_r) plus the mean EM
// terms X = eps0 <E_a E_b + c^2 B_a B_b>, Y = eps0 c <B x E> for f and g, and
// the Maxwell equilibrium of (Er, Br) = (<E>, <B>), J = 0, rho_c = 0 for h
void set_reference(RunState& r, const double* means)
{
    for (int j = 0; j < lb::NMEANS; ++j) r.means[j] = means[j];
    const double c = r.p.c, c2 = c * c, eps0 = 1.0 / c2;
    const double n_r = means[0], p_r = means[1];
    r.ref.n_r = n_r;
    r.ref.p_r = p_r;
    r.ref.eps_r = n_r * c2 + p_r / (r.p.gamma_ad - 1.0);
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int a = 0; a < 3; ++a) {
        r.Er[a] = means[2 + a];
        r.Br[a] = means[5 + a];
        r.Yr[a] = eps0 * c * means[20 + a];
    }
    for (int m = 0; m < 6; ++m) {
        const double x = eps0 * (means[8 + m] + c2 * means[14 + m]);
        r.Xr[ia[m]][ib[m]] = r.Xr[ib[m]][ia[m]] = x;
    }
    const double* Er = r.Er;
    const double* Br = r.Br;
    for (int kk = 0; kk < 24; ++kk) {
        const int p = kk / 8, i = (kk % 8) / 2, j = kk % 2, ie = (i + 3) % 4;
        const int a1 = lb::plane_a1(p), a2 = lb::plane_a2(p);
        const double e = lb::kSqrt2 / (16.0 * c) * (lb::hop_s1(ie) * Er[a1] + lb::hop_s2(ie) * Er[a2]);
        const double m = 0.125 * lb::plane_orient(p) * Br[lb::plane_normal(p)];
        r.refpops.h[kk] = j == 0 ? e - m : m - e;
    }
    r.refpops.h[24] = 0.0;
    const double tr = r.Xr[0][0] + r.Xr[1][1] + r.Xr[2][2];
    double fmax = 0.0, gmax = 0.0;
    for (int i = 0; i < 19; ++i) {
        const int cx = lb::c19(i, 0), cy = lb::c19(i, 1), cz = lb::c19(i, 2);
        double v = 3.0 * p_r;
        if (i == 0) v += lb::kRest * (3.0 * p_r - r.ref.eps_r);
        v += 2.3 * tr - lb::kSqrt19_3 * (cx * r.Yr[0] + cy * r.Yr[1] + cz * r.Yr[2]) -
             3.8 * (cx * cx * r.Xr[0][0] + cy * cy * r.Xr[1][1] + cz * cz * r.Xr[2][2]) -
             14.25 * (cx * cy * r.Xr[0][1] + cx * cz * r.Xr[0][2] + cy * cz * r.Xr[1][2]);
        r.refpops.f[i] = lb::w19(i) * v;
        r.refpops.g[i] = lb::wg19(i) * n_r;
        fmax = std::fmax(fmax, std::fabs(r.refpops.f[i]));
        gmax = std::fmax(gmax, std::fabs(r.refpops.g[i]));
    }
    for (int i = 0; i < 19; ++i) {
        if (r.p.precision == LBRMHD_FP16_DEV) {
            const double sf = std::fmax(std::fabs(r.refpops.f[i]), 0.05 * fmax);
            const double sg = std::fmax(std::fabs(r.refpops.g[i]), 0.05 * gmax);
            r.hs.f[i] = (float)sf;
            r.hs.finv[i] = (float)(1.0 / sf);
            r.hs.g[i] = (float)sg;
            r.hs.ginv[i] = (float)(1.0 / sg);
        } else {
            r.hs.f[i] = r.hs.finv[i] = r.hs.g[i] = r.hs.ginv[i] = 1.0f;
        }
    }
}

int ensure_io(lbrmhd_handle h, size_t bytes)
{
    if (h->io_bytes >= bytes) return LBRMHD_OK;
    if (h->d_io) cudaFree(h->d_io);
    h->d_io = nullptr;
    h->io_bytes = 0;
    if (cudaMalloc(&h->d_io, bytes) != cudaSuccess) return fail(h, LBRMHD_ERR_OOM, "staging allocation failed");
    h->io_bytes = bytes;
    return LBRMHD_OK;
}

int run_seed(const RunState& r)
{
    return r.p.recovery == LBRMHD_RECOVERY_MLP ? lb::SEED_MLP
           : (r.p.recovery == LBRMHD_RECOVERY_COLD || r.d_samples) ? lb::SEED_COLD
                                                                   : lb::SEED_PREV;
}

bool has_open(const RunState& r)
{
    return r.p.bc[0] || r.p.bc[1] || r.p.bc[2] || r.p.bc[3] || r.p.bc[4] || r.p.bc[5];
}

bool forced(const RunState& r) { return r.p.drive_f0 != 0.0 && r.p.drive_layers > 0; }
bool capped(const RunState& r) { return forced(r) && r.p.drive_vmax > 0.0; }

// runs stepped by the kernel variant with the open-face code (which also
// holds the body force)
bool open_variant(const RunState& r) { return has_open(r) || forced(r); }

// ---------------------------------------------------------------------------
// Tensor maps of the TMA tile kernel (2-D runs with periodic faces, float32 or
// float16 storage, rows a whole number of 16-byte units long)
// ---------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// whether a run's layout admits the tile kernel (the flags are checked at launch)
bool tile_layout_ok(const lbrmhd_params& p, bool open_var)
{
    if (p.precision == LBRMHD_FP64 || p.nz != 1 || open_var) return false;
    const int px = lb::tile_halo_x((int)pop_bytes(p.precision));
    return p.nx % px == 0 && p.nx >= lb::kTileW + 2 * px && p.ny >= lb::kTileH + 2 * lb::kTileHaloY;
}

// encodes one map of `rank` dims over `base`: rows of `vec` x nx elements
// (vec values per cell), ny rows, then `planes` planes of `vec` x stride
// elements; false if the driver rejects it
bool encode_map(CUtensorMap* m, CUtensorMapDataType dt, int elem, void* base, int rank, const RunState& r, int vec,
                int planes, const cuuint32_t* box)
{
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)vec * r.p.nx, (cuuint64_t)r.p.ny, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)vec * r.p.nx * elem, (cuuint64_t)vec * r.stride * elem};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, (cuuint32_t)rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the maps of both input buffers of a run (left empty where the tile kernel does not apply)
void make_tile_maps(RunState& r, int run_index)
{
    r.tmaps.clear();
    if (!tile_layout_ok(r.p, open_variant(r))) return;
    const int pb = (int)pop_bytes(r.p.precision);
    const int px = lb::tile_halo_x(pb), pxh = lb::tile_halo_x(4);
    const CUtensorMapDataType pdt = pb == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapDataType fdt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint32_t bh = lb::kTileH + 2 * lb::kTileHaloY;
    const cuuint32_t bwf = lb::kTileW + 2 * px, bwh = lb::kTileW + 2 * pxh;
    const cuuint32_t box_fg[3] = {4 * bwf, bh, 1};
    const cuuint32_t box_r[2] = {2 * bwf, bh};
    const cuuint32_t box_h[3] = {2 * bwh, bh, 2};
    const cuuint32_t box_h24[2] = {bwh, bh};
    const cuuint32_t box_p[3] = {4 * lb::kTileW, lb::kTileH, (cuuint32_t)lb::kPrimVecs};
    std::vector<lb::TileMaps> maps(2);
    bool ok = true;
    for (int in = 0; in < 2 && ok; ++in) {
        const int out = 1 - in;
        lb::TileMaps& m = maps[in];
        char* fg = (char*)r.pops[in];
        char* hh = (char*)r.h[in];
        ok = ok && encode_map(&m.fg_in, pdt, pb, fg, 3, r, 4, lb::kFGroups, box_fg);
        ok = ok && encode_map(&m.r_in, pdt, pb, fg + lb::fg_elem(0, 0, 0, r.stride) * pb, 2, r, 2, 1, box_r);
        ok = ok && encode_map(&m.h_in, fdt, 4, hh, 3, r, 2, 12, box_h);
        ok = ok && encode_map(&m.h24_in, fdt, 4, hh + lb::h_elem(24, 0, r.stride) * 4, 2, r, 1, 1, box_h24);
        ok = ok && encode_map(&m.p_in, fdt, 4, r.prim[in], 3, r, 4, lb::kPrimVecs, box_p);
        ok = ok && encode_map(&m.p_out, fdt, 4, r.prim[out], 3, r, 4, lb::kPrimVecs, box_p);
    }
    if (!ok) return;
    // the 32 x 4 tiles outside the rectangle of interior tiles, as (run, x0, y0, 0)
    const lb::TileRange tr = lb::interior_tiles(r.p.nx, r.p.ny, px);
    const int ix0 = tr.x0 * lb::kTileW, ix1 = (tr.x0 + tr.nx) * lb::kTileW;
    const int iy0 = tr.y0 * lb::kTileH, iy1 = (tr.y0 + tr.ny) * lb::kTileH;
    std::vector<int4> edge;
    for (int y0 = 0; y0 < r.p.ny; y0 += 4)
        for (int x0 = 0; x0 < r.p.nx; x0 += 32)
            if (!(x0 >= ix0 && x0 < ix1 && y0 >= iy0 && y0 < iy1)) edge.push_back(make_int4(run_index, x0, y0, 0));
    if (!edge.empty()) {
        if (cudaMalloc(&r.d_edge, edge.size() * sizeof(int4)) != cudaSuccess ||
            cudaMemcpy(r.d_edge, edge.data(), edge.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            if (r.d_edge) cudaFree(r.d_edge);
            r.d_edge = nullptr;
            return;
        }
    }
    r.nedge = (int)edge.size();
    r.tmaps = std::move(maps);
}


// kernel arguments of one run reading input buffer `in`
template <class Cfg>
lb::StepArgs<Cfg> make_args(lbrmhd_handle h, const RunState& r, int in)
{
    using R = typename Cfg::real;
    lb::StepArgs<Cfg> A{};
    const int out = 1 - in;
    A.fgin = (const typename Cfg::pop*)r.pops[in];
    A.hin = (const typename Cfg::hpop*)r.h[in];
    A.pin = (const typename Cfg::prim*)r.prim[in];
    A.fgout = (typename Cfg::pop*)r.pops[out];
    A.hout = (typename Cfg::hpop*)r.h[out];
    A.pout = (typename Cfg::prim*)r.prim[out];
    A.nx = r.p.nx;
    A.ny = r.p.ny;
    A.nz = r.p.nz;
    A.stride = r.stride;
    for (int a = 0; a < 3; ++a) A.periodic[a] = r.periodic[a];
    A.open_mask = 0;
    for (int a = 0; a < 3; ++a)
        if (r.p.bc[2 * a] != 0 || r.p.bc[2 * a + 1] != 0) A.open_mask |= 1 << a;
    A.flags = r.p.flags;
    A.k = make_phys<R>(r.p, r.ref, runref(r));
    A.hs = r.hs;
    A.stats = r.d_stats;
    A.mlp = h->d_mlp;
    A.dump = r.d_samples;
    A.seed = run_seed(r);
    A.status = h->d_status;
    if (forced(r)) {
        const double dt = r.p.dx / (std::sqrt(2.0) * r.p.c);
        A.open_mask |= lb::OPEN_EXTRA;
        A.fdrive = r.d_drive;
        A.force_layers = std::min(r.p.drive_layers, r.p.nz);
        A.vmax2 = capped(r) ? r.p.drive_vmax * r.p.drive_vmax : 0.0;
        A.umax_in = r.d_umax;
        A.umax_out = capped(r) ? r.d_umax + 1 : nullptr;
        A.force_cdt = (R)(r.p.c * dt / (10.0 * lb::kQ));
        A.force_dt = (R)dt;
    }
    return A;
}

// whether the per-run launch covers run r: its grid is (nx / bx) x (ny x bx / 128)
// x nz blocks with bx <= 128, and a grid's y and z extents are limited to 65535
bool per_run_launchable(const RunState& r) { return r.p.ny <= 65535 && r.p.nz <= 65535; }

// the schedule the steps run with: the one set, except that a PER_RUN schedule
// of a handle with a run the per-run launch cannot cover walks the tile list
// (BATCH, 128-wide tiles, one wave of resident blocks) for every run
lbrmhd_schedule effective_schedule(lbrmhd_handle h)
{
    lbrmhd_schedule s = h->sched;
    if (s.kind != LBRMHD_SCHED_PER_RUN) return s;
    for (const auto& r : h->runs)
        if (!per_run_launchable(r)) {
            s.kind = LBRMHD_SCHED_BATCH;
            s.bx = 128;
            s.waves = 1;
            s.order = 0;
            s.streams = 1;
            break;
        }
    return s;
}

// tile list of the batched schedule, grouped by kernel variant (2-D / 3-D,
// recovery seed); within a group tiles follow the runs in order (order 0) or
// are interleaved across runs (order 1)
int build_tiles(lbrmhd_handle h, const lbrmhd_schedule& sc)
{
    const int bx = sc.bx, by = lb::kStepThreads / sc.bx;
    std::vector<int4> all;
    h->groups.clear();
    for (int is3d = 0; is3d < 2; ++is3d)
        for (int seed = 0; seed < 3; ++seed)
        for (int open = 0; open < 2; ++open) {
            std::vector<std::vector<int4>> per;
            for (int ri = 0; ri < (int)h->runs.size(); ++ri) {
                const RunState& r = h->runs[ri];
                if ((r.p.nz > 1) != (is3d == 1) || run_seed(r) != seed || open_variant(r) != (open == 1)) continue;
                std::vector<int4> t;
                for (int z = 0; z < r.p.nz; ++z)
                    for (int y0 = 0; y0 < r.p.ny; y0 += by)
                        for (int x0 = 0; x0 < r.p.nx; x0 += bx) t.push_back(make_int4(ri, x0, y0, z));
                per.push_back(std::move(t));
            }
            if (per.empty()) continue;
            const int first = (int)all.size();
            if (sc.order == 0) {
                for (auto& t : per) all.insert(all.end(), t.begin(), t.end());
            } else {
                size_t longest = 0;
                for (auto& t : per) longest = std::max(longest, t.size());
                for (size_t i = 0; i < longest; ++i)
                    for (auto& t : per)
                        if (i < t.size()) all.push_back(t[i]);
            }
            h->groups.push_back({is3d == 1, open == 1, seed, first, (int)all.size() - first});
        }
    if (all.size() > (size_t)0x7fffffff) return fail(h, LBRMHD_ERR_BAD_ARG, "too many tiles for one launch");
    if (all.size() > h->tiles_cap) {
        if (h->d_tiles) cudaFree(h->d_tiles);
        h->d_tiles = nullptr;
        h->tiles_cap = 0;
        if (cudaMalloc(&h->d_tiles, all.size() * sizeof(int4)) != cudaSuccess)
            return fail(h, LBRMHD_ERR_OOM, "tile list allocation failed");
        h->tiles_cap = all.size();
    }
    LB_CK(cudaMemcpy(h->d_tiles, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice));
    h->tiles_dirty = false;
    return LBRMHD_OK;
}

template <class Cfg>
int upload_args(lbrmhd_handle h)
{
    const size_t n = h->runs.size(), stride = lb::batch_args_stride<Cfg>();
    std::vector<unsigned char> a(2 * n * stride, 0);
    for (int in = 0; in < 2; ++in)
        for (size_t ri = 0; ri < n; ++ri) {
            const lb::StepArgs<Cfg> A = make_args<Cfg>(h, h->runs[ri], in);
            std::memcpy(a.data() + (in * n + ri) * stride, &A, sizeof(A));
        }
    if (!h->d_args && cudaMalloc(&h->d_args, a.size()) != cudaSuccess) {
        h->d_args = nullptr;
        return fail(h, LBRMHD_ERR_OOM, "argument array allocation failed");
    }
    LB_CK(cudaMemcpy(h->d_args, a.data(), a.size(), cudaMemcpyHostToDevice));
    h->args_dirty = false;
    return LBRMHD_OK;
}

// the tiled launch of run `ri` from input buffer `in` (NULL: the per-cell kernel)
template <class Cfg>
bool tile_launch(lbrmhd_handle h, size_t ri, int in, lb::TileLaunch* tl)
{
    const RunState& r = h->runs[ri];
    if (r.tmaps.empty()) return false;
    tl->maps = &r.tmaps[in];
    tl->args = (const unsigned char*)h->d_args + (size_t)in * h->runs.size() * lb::batch_args_stride<Cfg>();
    tl->edge_tiles = r.d_edge;
    tl->nedge = r.nedge;
    tl->sms = h->sms;
    return true;
}

// everything a batched launch needs, refreshed when the runs or the schedule
// changed (the tiled per-run launch reads its edge runs' arguments from the
// same device records)
template <class Cfg>
int prepare_batch(lbrmhd_handle h, const lbrmhd_schedule& sc)
{
    bool tiled = false;
    for (const auto& r : h->runs) tiled = tiled || !r.tmaps.empty();
    if (sc.kind == LBRMHD_SCHED_PER_RUN) return tiled && h->args_dirty ? upload_args<Cfg>(h) : LBRMHD_OK;
    int rc = LBRMHD_OK;
    if (h->tiles_dirty) rc = build_tiles(h, sc);
    if (!rc && h->args_dirty) rc = upload_args<Cfg>(h);
    return rc;
}

// one time step of every run reading input buffer `in` (the same for all
// runs), issued on stream `s`; the host state (cur, step counters) is not
// touched, so a caller can also issue a dry step whose output is discarded
template <class Cfg>
int issue_step(lbrmhd_handle h, const lbrmhd_schedule& sc, int in, cudaStream_t s)
{
    using R = typename Cfg::real;
    const int out = 1 - in;
    if (sc.kind == LBRMHD_SCHED_BATCH) {
        const unsigned char* args = (const unsigned char*)h->d_args + (size_t)in * h->runs.size() * lb::batch_args_stride<Cfg>();
        int dev_sms = 0;
        LB_CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device));
        for (const auto& g : h->groups) {
            int grid = 0;  // one block per tile
            if (sc.waves > 0)
                grid = sc.waves * dev_sms * std::max(1, lb::batch_blocks_per_sm<Cfg>(g.is3d, g.seed, g.open));
            LB_CK(lb::launch_step_batch<Cfg>(args, h->d_tiles + g.first, g.count, sc.bx, grid, g.is3d, g.seed, g.open,
                                             s));
        }
    } else {
        for (size_t ri = 0; ri < h->runs.size(); ++ri) {
            lb::TileLaunch tl{};
            const bool t = tile_launch<Cfg>(h, ri, in, &tl);
            LB_CK(lb::launch_step<Cfg>(make_args<Cfg>(h, h->runs[ri], in), s, t ? &tl : nullptr));
        }
    }
    for (const auto& r : h->runs) {
        if (has_open(r))
            LB_CK(lb::launch_boundaries<Cfg>(view<Cfg>(r, out), make_phys<R>(r.p, r.ref, runref(r)), r.p.bc,
                                             r.p.drive_layers, r.d_drive, s));
        if (capped(r)) LB_CK(lb::launch_umax_roll(r.d_umax, s));
    }
    return LBRMHD_OK;
}

int ensure_aux(lbrmhd_handle h, int n)
{
    if (!h->ev_fork) LB_CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    while ((int)h->aux.size() < n) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        LB_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        h->aux.push_back(st);
        LB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->aux_join.push_back(ev);
    }
    return LBRMHD_OK;
}

// whether the handle's runs admit the persistent launch: every run periodic
// and unforced (no boundary or cut-off pass between steps) and all of one
// kernel variant
std::string persistent_unsupported(lbrmhd_handle h)
{
    for (const auto& r : h->runs)
        if (open_variant(r) || capped(r)) return "the persistent schedule needs periodic, unforced runs";
    for (const auto& r : h->runs)
        if ((r.p.nz > 1) != (h->runs[0].p.nz > 1) || run_seed(r) != run_seed(h->runs[0]))
            return "the persistent schedule needs runs of one kernel variant (all 2-D or all 3-D, one seed)";
    return "";
}

constexpr unsigned long long kBarrierWaitNs = 1000ull * 1000ull * 1000ull;  // 1 s

// n steps of every run in one cooperative launch (tiles and arguments prepared)
template <class Cfg>
int issue_persistent(lbrmhd_handle h, const lbrmhd_schedule& sc, int in, int64_t n, cudaStream_t s)
{
    const std::string m = persistent_unsupported(h);
    if (!m.empty()) return fail(h, LBRMHD_ERR_BAD_ARG, m);
    if (h->groups.size() != 1) return fail(h, LBRMHD_ERR_STATE, "persistent launch needs one tile group");
    const auto& g = h->groups[0];
    int dev_sms = 0;
    LB_CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device));
    const int per_sm = lb::persistent_blocks_per_sm<Cfg>(g.is3d, g.seed, g.open);
    if (per_sm < 1) return fail(h, LBRMHD_ERR_CUDA, "persistent kernel does not fit on an SM");
    const int grid = std::min(per_sm * dev_sms, g.count);
    const size_t parity_bytes = h->runs.size() * lb::batch_args_stride<Cfg>();
    for (int64_t done = 0; done < n;) {
        const int k = (int)std::min<int64_t>(n - done, 1 << 20);
        LB_CK(cudaMemsetAsync(h->d_barrier, 0, sizeof(unsigned int), s));
        LB_CK(lb::launch_step_persistent<Cfg>((const unsigned char*)h->d_args, parity_bytes, (int)((in + done) & 1),
                                              h->d_tiles + g.first, g.count, sc.bx, k, grid, g.is3d, g.seed, g.open,
                                              h->d_barrier, h->d_status, kBarrierWaitNs, s));
        done += k;
    }
    return LBRMHD_OK;
}

// n steps of every run from input buffer `in`, issued after and completed
// before the work of stream `s` (host state untouched, as issue_step)
template <class Cfg>
int issue_steps(lbrmhd_handle h, const lbrmhd_schedule& sc, int in, int64_t n, cudaStream_t s)
{
    using R = typename Cfg::real;
    if (sc.kind == LBRMHD_SCHED_PERSISTENT) return issue_persistent<Cfg>(h, sc, in, n, s);
    const int S = sc.kind == LBRMHD_SCHED_PER_RUN ? std::min<int>(sc.streams, (int)h->runs.size()) : 1;
    if (S <= 1) {
        for (int64_t t = 0; t < n; ++t) {
            const int rc = issue_step<Cfg>(h, sc, (int)((in + t) & 1), s);
            if (rc) return rc;
        }
        return LBRMHD_OK;
    }
    int rc = ensure_aux(h, S);
    if (rc) return rc;
    LB_CK(cudaEventRecord(h->ev_fork, s));
    for (int i = 0; i < S; ++i) LB_CK(cudaStreamWaitEvent(h->aux[i], h->ev_fork, 0));
    for (int64_t t = 0; t < n; ++t) {
        const int cin = (int)((in + t) & 1);
        for (size_t ri = 0; ri < h->runs.size(); ++ri) {
            const RunState& r = h->runs[ri];
            cudaStream_t st = h->aux[ri % S];
            lb::TileLaunch tl{};
            const bool t = tile_launch<Cfg>(h, ri, cin, &tl);
            LB_CK(lb::launch_step<Cfg>(make_args<Cfg>(h, r, cin), st, t ? &tl : nullptr));
            if (has_open(r))
                LB_CK(lb::launch_boundaries<Cfg>(view<Cfg>(r, 1 - cin), make_phys<R>(r.p, r.ref, runref(r)), r.p.bc,
                                                 r.p.drive_layers, r.d_drive, st));
            if (capped(r)) LB_CK(lb::launch_umax_roll(r.d_umax, st));
        }
    }
    for (int i = 0; i < S; ++i) {
        LB_CK(cudaEventRecord(h->aux_join[i], h->aux[i]));
        LB_CK(cudaStreamWaitEvent(s, h->aux_join[i], 0));
    }
    return LBRMHD_OK;
}

void drop_graphs(lbrmhd_handle h)
{
    for (auto& g : h->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    h->graph_len = 0;
}

// the runs' state changed (init, checkpoint, sample buffer): arguments and graphs are stale
void runs_changed(lbrmhd_handle h)
{
    h->args_dirty = true;
    h->tiles_dirty = true;  // a sample buffer can move a run to another kernel variant
    drop_graphs(h);
}

template <class Cfg>
int capture_graph(lbrmhd_handle h, const lbrmhd_schedule& sc, int in)
{
    if (!h->cap_stream) {
        LB_CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        LB_CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
        LB_CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    }
    for (const auto& g : h->groups) lb::batch_blocks_per_sm<Cfg>(g.is3d, g.seed, g.open);  // attributes set before capture
    if (sc.kind == LBRMHD_SCHED_PER_RUN && sc.streams > 1) {
        const int rc0 = ensure_aux(h, std::min<int>(sc.streams, (int)h->runs.size()));  // created outside the capture
        if (rc0) return rc0;
    }
    LB_CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = issue_steps<Cfg>(h, sc, in, sc.graph_steps, h->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(h, LBRMHD_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&h->graph[in], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        h->graph[in] = nullptr;
        return fail(h, LBRMHD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    h->graph_len = sc.graph_steps;
    return LBRMHD_OK;
}

// n steps of every run; whole graphs first (when enabled), then direct launches
template <class Cfg>
int step_all(lbrmhd_handle h, int64_t n)
{
    const lbrmhd_schedule sc = effective_schedule(h);
    int rc = prepare_batch<Cfg>(h, sc);
    if (rc) return rc;
    int in = h->runs[0].cur;
    int64_t done = 0;
    if (sc.graph_steps > 0 && n >= sc.graph_steps) {
        if (h->graph_len != sc.graph_steps) drop_graphs(h);
        if (!h->graph[in]) rc = capture_graph<Cfg>(h, sc, in);
        if (rc) return rc;
        LB_CK(cudaEventRecord(h->ev_in, h->stream));
        LB_CK(cudaStreamWaitEvent(h->cap_stream, h->ev_in, 0));
        for (; done + sc.graph_steps <= n; done += sc.graph_steps) {
            if (!h->graph[in]) {
                rc = capture_graph<Cfg>(h, sc, in);
                if (rc) return rc;
            }
            LB_CK(cudaGraphLaunch(h->graph[in], h->cap_stream));
            in = (in + sc.graph_steps) & 1;
        }
        LB_CK(cudaEventRecord(h->ev_out, h->cap_stream));
        LB_CK(cudaStreamWaitEvent(h->stream, h->ev_out, 0));
    }
    if (done < n) {
        rc = issue_steps<Cfg>(h, sc, in, n - done, h->stream);
        if (rc) return rc;
        in = (int)((in + (n - done)) & 1);
    }
    for (auto& r : h->runs) {
        r.cur = in;
        r.steps += n;
    }
    return LBRMHD_OK;
}

template <class Cfg>
int init_run(lbrmhd_handle h, RunState& r, const lb::InitInputs& in)
{
    LB_CK(lb::launch_means(in, r.N, h->d_scratch, h->d_small, h->stream));
    double mean[lb::NMEANS];
    LB_CK(cudaMemcpyAsync(mean, h->d_small, sizeof(mean), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    set_reference(r, mean);
    LB_CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LB_CK(lb::launch_init<Cfg>(view<Cfg>(r, r.cur), in, make_phys<double>(r.p, r.ref, runref(r)), h->d_flag, h->stream));
    int bad = 0;
    LB_CK(cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaMemsetAsync(r.d_stats, 0, kStatsAlloc, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    if (bad) return fail(h, LBRMHD_ERR_BAD_ARG, "initial state has |u| >= c or n <= 0");
    LB_CK(lb::launch_prim_component<Cfg>(view<Cfg>(r, r.cur), lb::P_E + 2, (typename Cfg::prim*)r.d_ez0, h->stream));
    if (capped(r)) LB_CK(lb::launch_umax_state<Cfg>(view<Cfg>(r, r.cur), r.d_umax, h->stream));
    r.initialized = true;
    runs_changed(h);
    r.steps = 0;
    return LBRMHD_OK;
}

// the cut-off's maximum |u|^2 taken from the current state of a run
int refresh_umax(lbrmhd_handle h, RunState& r)
{
    if (!capped(r)) return LBRMHD_OK;
    switch (h->precision) {
        case LBRMHD_FP64: LB_CK(lb::launch_umax_state<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), r.d_umax, h->stream)); break;
        case LBRMHD_FP32: LB_CK(lb::launch_umax_state<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), r.d_umax, h->stream)); break;
        default: LB_CK(lb::launch_umax_state<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), r.d_umax, h->stream));
    }
    return LBRMHD_OK;
}

int init_common(lbrmhd_handle h, int run, const double* n, const double* p, const double* u, const double* B,
                const double* E, bool device_inputs)
{
    if (bad_run(h, run)) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "run out of range") : LBRMHD_ERR_BAD_ARG;
    if (!n || !p || !u || !B) return fail(h, LBRMHD_ERR_BAD_ARG, "NULL input array");
    LB_CK(cudaSetDevice(h->device));
    RunState& r = h->runs[run];
    const int64_t N = r.N;
    lb::InitInputs in{};
    if (device_inputs) {
        in = {n, p, u, B, E};
    } else {
        int rc = ensure_io(h, (size_t)11 * N * sizeof(double));
        if (rc) return rc;
        double* d = h->d_io;
        LB_CK(cudaMemcpyAsync(d, n, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(d + N, p, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(d + 2 * N, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(d + 5 * N, B, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if (E) LB_CK(cudaMemcpyAsync(d + 8 * N, E, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        in = {d, d + N, d + 2 * N, d + 5 * N, E ? d + 8 * N : nullptr};
    }
    switch (h->precision) {
        case LBRMHD_FP64: return init_run<lb::CfgF64>(h, r, in);
        case LBRMHD_FP32: return init_run<lb::CfgF32>(h, r, in);
        default: return init_run<lb::CfgF16>(h, r, in);
    }
}

std::string check_params(const lbrmhd_params& p)
{
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return "grid sizes must be >= 1";
    // the step kernel forms its stencil offsets (up to the periodic wrap, ~N
    // cells) in 32 bits and scales them by the 4-wide population groups
    if ((int64_t)p.nx * p.ny * p.nz > ((int64_t)1 << 29)) return "grid too large (more than 2^29 cells)";
    if (!(p.c > 0) || !(p.dx > 0) || !(p.tau > 0)) return "c, dx and tau must be > 0";
    if (!(p.sigma >= 0)) return "sigma must be >= 0";
    if (!(p.gamma_ad > 1)) return "gamma_ad must be > 1";
    if (!(p.alpha >= 0)) return "alpha must be >= 0";
    if (p.precision < LBRMHD_FP64 || p.precision > LBRMHD_FP16_DEV) return "unknown precision";
    if (p.recovery != LBRMHD_RECOVERY_PLAIN && p.recovery != LBRMHD_RECOVERY_MLP && p.recovery != LBRMHD_RECOVERY_COLD)
        return "unknown recovery mode";
    if (p.flags & ~(LBRMHD_FLAG_NO_EM_COLLISION | LBRMHD_FLAG_UNSHIFTED_POWER | LBRMHD_FLAG_ONE_PASS_RECOVERY |
                    LBRMHD_FLAG_GAUSS_CHARGE | LBRMHD_FLAG_TMA_TILES | LBRMHD_FLAG_FIRST_ORDER_FLUX))
        return "unknown flag";
    for (int f = 0; f < 6; ++f) {
        if (p.bc[f] < 0 || p.bc[f] > 2) return "unknown boundary kind";
        if (p.bc[f] == LBRMHD_DRIVEN && f != 4) return "DRIVEN is only allowed on the -z face";
    }
    for (int a = 0; a < 3; ++a)
        if ((p.bc[2 * a] == LBRMHD_PERIODIC) != (p.bc[2 * a + 1] == LBRMHD_PERIODIC))
            return "an axis must be periodic on both faces or on neither";
    if (p.bc[4] == LBRMHD_DRIVEN && p.drive_layers < 0) return "drive_layers must be >= 0";
    if (!std::isfinite(p.drive_f0) || !std::isfinite(p.drive_vmax)) return "drive_f0 and drive_vmax must be finite";
    if (p.drive_f0 != 0.0) {
        if (p.drive_layers < 1) return "a body force needs drive_layers >= 1";
        if (p.bc[4] == LBRMHD_DRIVEN) return "a body force replaces the DRIVEN face: use OPEN or PERIODIC on -z";
    }
    return "";
}

// ---------------------------------------------------------------------------
// Scratch for lbrmhd_get_diagnostics_noalloc: a fixed, file-scope device array
// instead of any allocation. It holds the per-block partial sums of the
// diagnostics reduction (NPART float64 per block of kDiagThreads cells), for
// at most kNoAllocMaxBlocks blocks, i.e. runs of up to
// kNoAllocMaxBlocks * kDiagThreads = 16,777,216 cells (256^3): 4.7 MB that every
// GPU that loads this library keeps until the process exits.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxBlocks = 65536;
constexpr int64_t kNoAllocMaxCells = kNoAllocMaxBlocks * lb::kDiagThreads;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * lb::NPART];

// The host-side name g_noalloc_partials is only a stand-in for the device
// array, not its address; a kernel handed it would fault or, on systems where
// the GPU can reach host memory, silently use the wrong memory. lbrmhd_create
// looks the device address up with the handle's device current and keeps it
// in the handle, so the address always belongs to the context the handle's
// kernels run in (nothing is cached across handles or contexts).
int lookup_noalloc_scratch(double** out)
{
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        *out = nullptr;
        return LBRMHD_ERR_CUDA;
    }
    *out = p;
    return LBRMHD_OK;
}

// totals of the per-slot recovery counters of one run (synchronises the stream)
int read_stats(lbrmhd_handle h, const RunState& r, unsigned long long* tot)
{
    std::vector<unsigned long long> all((size_t)lb::kStatSlots * lb::kNumStats);
    LB_CK(cudaMemcpyAsync(all.data(), r.d_stats, kStatsAlloc, cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < lb::kNumStats; ++i) tot[i] = 0;
    for (int sl = 0; sl < lb::kStatSlots; ++sl) {
        const unsigned long long* v = all.data() + (size_t)sl * lb::kNumStats;
        for (int i = 0; i < lb::kNumStats; ++i) tot[i] = i == 2 ? std::max(tot[i], v[i]) : tot[i] + v[i];
    }
    return LBRMHD_OK;
}

// writes checkpointed totals back: slot 0 holds them, the other slots zero
int write_stats(lbrmhd_handle h, const RunState& r, const unsigned long long* tot)
{
    LB_CK(cudaMemsetAsync(r.d_stats, 0, kStatsAlloc, h->stream));
    LB_CK(cudaMemcpyAsync(r.d_stats, tot, kStatsBytes, cudaMemcpyHostToDevice, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

std::string check_schedule(const lbrmhd_schedule& s)
{
    if (s.kind != LBRMHD_SCHED_PER_RUN && s.kind != LBRMHD_SCHED_BATCH && s.kind != LBRMHD_SCHED_PERSISTENT)
        return "unknown schedule kind";
    if (s.bx != 32 && s.bx != 64 && s.bx != 128) return "tile width must be 32, 64 or 128";
    if (s.waves < 0 || s.waves > 8) return "waves must be in 0..8";
    if (s.order != 0 && s.order != 1) return "order must be 0 or 1";
    if (s.streams < 1 || s.streams > 32) return "streams must be in 1..32";
    if (s.graph_steps < 0 || s.graph_steps > 4096) return "graph_steps must be in 0..4096";
    return "";
}

// key of a batch for the autotuner cache: precision and, per run, the grid
// and the kernel variant
std::string batch_signature(lbrmhd_handle h)
{
    std::ostringstream o;
    o << "p" << h->precision;
    for (const auto& r : h->runs)
        o << "_" << r.p.nx << "x" << r.p.ny << "x" << r.p.nz << "s" << run_seed(r) << (open_variant(r) ? "o" : "");
    return o.str();
}

bool cache_lookup(const std::string& path, const std::string& sig, lbrmhd_schedule* sc, double* ms)
{
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {  // the last entry of a signature wins
        std::istringstream in(line);
        std::string key;
        lbrmhd_schedule c{};
        double t = 0;
        if (in >> key >> c.kind >> c.bx >> c.waves >> c.order >> c.streams >> t && key == sig &&
            check_schedule(c).empty()) {
            *sc = c;
            *ms = t;
            found = true;
        }
    }
    return found;
}

template <class Cfg>
int autotune(lbrmhd_handle h, int trials, lbrmhd_schedule* best_out, double* best_ms_out)
{
    for (auto& r : h->runs) {
        if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "autotune before lbrmhd_init_fields");
        if (r.p.recovery == LBRMHD_RECOVERY_MLP && !h->mlp_set)
            return fail(h, LBRMHD_ERR_STATE, "learned-seed run without weights (lbrmhd_set_mlp_weights)");
        if (r.cur != h->runs[0].cur) return fail(h, LBRMHD_ERR_STATE, "runs out of step");
    }
    const lbrmhd_schedule cur = effective_schedule(h);
    const char* cache = std::getenv("LBRMHD_TUNE_CACHE");
    const std::string sig = batch_signature(h);
    lbrmhd_schedule best = cur;
    double best_ms = -1.0;
    if (!(cache && *cache && cache_lookup(cache, sig, &best, &best_ms))) {
        std::vector<lbrmhd_schedule> cand;
        const int nr = (int)h->runs.size();
        bool per_run = true;
        for (const auto& r : h->runs) per_run = per_run && per_run_launchable(r);
        if (per_run) {
            cand.push_back({LBRMHD_SCHED_PER_RUN, 128, 0, 0, 1, 0});
            if (nr > 1) cand.push_back({LBRMHD_SCHED_PER_RUN, 128, 0, 0, std::min(nr, 4), 0});
            if (nr > 4) cand.push_back({LBRMHD_SCHED_PER_RUN, 128, 0, 0, std::min(nr, 16), 0});
        }
        for (int bx : {128, 64, 32})
            for (int waves : {0, 1})
                for (int order : {0, 1})
                    if (nr > 1 || order == 0) cand.push_back({LBRMHD_SCHED_BATCH, bx, waves, order, 1, 0});
        if (persistent_unsupported(h).empty())
            for (int bx : {128, 64, 32})
                for (int order : {0, 1})
                    if (nr > 1 || order == 0) cand.push_back({LBRMHD_SCHED_PERSISTENT, bx, 1, order, 1, 0});
        // the counters are restored afterwards: dry steps only write the
        // scratch (output) buffers
        std::vector<std::vector<unsigned long long>> saved(h->runs.size(),
                                                           std::vector<unsigned long long>(lb::kNumStats));
        for (size_t i = 0; i < h->runs.size(); ++i) {
            const int rc = read_stats(h, h->runs[i], saved[i].data());
            if (rc) return rc;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        LB_CK(cudaEventCreate(&e0));
        LB_CK(cudaEventCreate(&e1));
        const int in = h->runs[0].cur;
        int rc = LBRMHD_OK;
        for (const auto& c : cand) {
            h->tiles_dirty = true;
            rc = prepare_batch<Cfg>(h, c);
            if (!rc) rc = issue_steps<Cfg>(h, c, in, 1, h->stream);  // warm-up (dry: the state stays at `in`)
            if (rc) break;
            if (cudaEventRecord(e0, h->stream) != cudaSuccess) rc = fail(h, LBRMHD_ERR_CUDA, "event record");
            for (int t = 0; t < trials && !rc; ++t) rc = issue_steps<Cfg>(h, c, in, 1, h->stream);
            if (!rc && cudaEventRecord(e1, h->stream) != cudaSuccess) rc = fail(h, LBRMHD_ERR_CUDA, "event record");
            if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(h, LBRMHD_ERR_CUDA, "autotune step failed");
            if (rc) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / trials;
            if (best_ms < 0 || per < best_ms) {
                best_ms = per;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (size_t i = 0; i < h->runs.size() && !rc; ++i) rc = write_stats(h, h->runs[i], saved[i].data());
        // the dry steps rolled the body-force cut-off's maximum: take it from the state again
        for (size_t i = 0; i < h->runs.size() && !rc; ++i) rc = refresh_umax(h, h->runs[i]);
        if (rc) return rc;
        if (cache && *cache) {
            std::ofstream f(cache, std::ios::app);
            f << sig << " " << best.kind << " " << best.bx << " " << best.waves << " " << best.order << " "
              << best.streams << " " << best_ms
              << "\n";
        }
    }
    best.graph_steps = cur.graph_steps;
    h->sched = best;
    h->tiles_dirty = true;
    drop_graphs(h);
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return LBRMHD_OK;
}

}  // namespace

namespace {

// The relaxed initialisation after init_common(host inputs): the inputs n, p,
// u (3), B (3) are in h->d_io, the layout the step kernel's relaxation reads.
template <class Cfg>
int relax_run(lbrmhd_handle h, RunState& r, int max_iters, double tol, int* iters, double* residual)
{
    using R = typename Cfg::real;
    const int64_t N = r.N;
    const int start = r.cur;
    double* e = nullptr;  // E_{k-1}, E_{k-2}
    if (cudaMalloc(&e, 6 * N * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, LBRMHD_ERR_OOM, "relaxation history allocation failed");
    }
    int k = 0;
    double res = 0.0;
    cudaError_t ce = lb::launch_relax_history<Cfg>(view<Cfg>(r, r.cur), e, h->stream);
    while (ce == cudaSuccess && k < max_iters) {
        ++k;
        ce = cudaMemsetAsync(h->d_small, 0, 2 * sizeof(double), h->stream);
        lb::StepArgs<Cfg> A = make_args<Cfg>(h, r, r.cur);
        A.force_layers = 0;  // no body force while the fields relax
        A.umax_out = nullptr;
        A.seed = lb::SEED_PREV;  // the plain open-face variant (the seed does not change the converged state)
        A.open_mask |= lb::OPEN_EXTRA;
        A.relax_in = h->d_io;
        A.relax_e = e;
        A.relax_red = h->d_small;
        if (ce == cudaSuccess) ce = lb::launch_step<Cfg>(A, h->stream, nullptr);
        if (ce == cudaSuccess && has_open(r))
            ce = lb::launch_boundaries<Cfg>(view<Cfg>(r, 1 - r.cur), make_phys<R>(r.p, r.ref, runref(r)), r.p.bc,
                                            r.p.drive_layers, r.d_drive, h->stream);
        r.cur ^= 1;
        double red[2] = {0.0, 0.0};
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(red, h->d_small, sizeof(red), cudaMemcpyDeviceToHost, h->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
        res = red[1] > 0.0 ? std::sqrt(red[0] / red[1]) : (red[0] > 0.0 ? INFINITY : 0.0);
        if (res <= tol) break;
    }
    cudaFree(e);
    if (ce != cudaSuccess) return fail(h, LBRMHD_ERR_CUDA, std::string("relaxed initialisation: ") + cudaGetErrorString(ce));
    // every run of a handle steps from the same buffer parity
    if (r.cur != start) {
        const size_t pb = pop_bytes(h->precision), hb = hp_bytes(h->precision);
        LB_CK(cudaMemcpyAsync(r.pops[start], r.pops[r.cur], 38 * r.stride * pb, cudaMemcpyDeviceToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(r.h[start], r.h[r.cur], 25 * r.stride * hb, cudaMemcpyDeviceToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(r.prim[start], r.prim[r.cur], lb::NPRIM * r.stride * hb, cudaMemcpyDeviceToDevice,
                              h->stream));
        r.cur = start;
    }
    // a fresh start: counters, step count, E^z_0, the cut-off's maximum
    LB_CK(cudaMemsetAsync(r.d_stats, 0, kStatsAlloc, h->stream));
    LB_CK(lb::launch_prim_component<Cfg>(view<Cfg>(r, r.cur), lb::P_E + 2, (typename Cfg::prim*)r.d_ez0, h->stream));
    if (capped(r)) LB_CK(lb::launch_umax_state<Cfg>(view<Cfg>(r, r.cur), r.d_umax, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    r.steps = 0;
    runs_changed(h);
    if (iters) *iters = k;
    if (residual) *residual = res;
    return LBRMHD_OK;
}

// The populations of a run's buffer as contiguous element ranges over its N
// cells (the padding of each plane left out): fluid, the nine group planes (4
// values per cell) and the rest pair; Maxwell, the twelve pairs and h_24.
struct Segment {
    int64_t first, count;
};
std::vector<Segment> state_segments(const RunState& r, bool fluid)
{
    std::vector<Segment> s;
    if (fluid) {
        for (int G = 0; G < lb::kFGroups; ++G) s.push_back({lb::fg_elem(2 * G + 1, 0, 0, r.stride), 4 * r.N});
        s.push_back({lb::fg_elem(0, 0, 0, r.stride), 2 * r.N});
    } else {
        for (int m = 0; m < 12; ++m) s.push_back({lb::h_elem(2 * m, 0, r.stride), 2 * r.N});
        s.push_back({lb::h_elem(24, 0, r.stride), r.N});
    }
    return s;
}

}  // namespace

extern "C" {

int lbrmhd_create(const lbrmhd_params* params, int n_runs, lbrmhd_handle* out)
{
    if (out) *out = nullptr;
    if (!params || n_runs < 1 || !out) {
        g_create_error = "NULL params / out or n_runs < 1";
        return LBRMHD_ERR_BAD_ARG;
    }
    for (int r = 0; r < n_runs; ++r) {
        std::string m = check_params(params[r]);
        if (m.empty() && params[r].precision != params[0].precision) m = "precision differs between runs";
        if (!m.empty()) {
            g_create_error = "run " + std::to_string(r) + ": " + m;
            return LBRMHD_ERR_BAD_ARG;
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        g_create_error = "no CUDA device available";
        return LBRMHD_ERR_CUDA;
    }
    lbrmhd_handle h = new lbrmhd_state_s();
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->sms < 1) h->sms = 1;
    h->precision = params[0].precision;
    const size_t pb = pop_bytes(h->precision), hb = hp_bytes(h->precision), qb = hp_bytes(h->precision);
    int64_t max_blocks = 1;
    bool ok = true;
    h->runs.resize(n_runs);
    for (int r = 0; r < n_runs && ok; ++r) {
        RunState& s = h->runs[r];
        s.p = params[r];
        s.N = (int64_t)s.p.nx * s.p.ny * s.p.nz;
        s.stride = (s.N + 127) / 128 * 128;
        for (int a = 0; a < 3; ++a) s.periodic[a] = s.p.bc[2 * a] == LBRMHD_PERIODIC;
        double m0[lb::NMEANS] = {1.0, 1.0};
        set_reference(s, m0);
        for (int b = 0; b < 2 && ok; ++b) {
            ok = ok && cudaMalloc(&s.pops[b], 38 * s.stride * pb) == cudaSuccess;
            ok = ok && cudaMalloc(&s.h[b], 25 * s.stride * hb) == cudaSuccess;
            ok = ok && cudaMalloc(&s.prim[b], lb::NPRIM * s.stride * qb) == cudaSuccess;
            if (ok) {
                cudaMemset(s.pops[b], 0, 38 * s.stride * pb);
                cudaMemset(s.h[b], 0, 25 * s.stride * hb);
                cudaMemset(s.prim[b], 0, lb::NPRIM * s.stride * qb);
            }
        }
        ok = ok && cudaMalloc(&s.d_ez0, s.N * qb) == cudaSuccess;
        if (ok && (s.p.bc[4] == LBRMHD_DRIVEN || forced(s))) {
            // the two-vortex pattern: velocity of the driven layers, or the force density
            const double amp = forced(s) ? s.p.drive_f0 : s.p.drive_u0;
            ok = cudaMalloc(&s.d_drive, 2 * sizeof(double) * s.p.nx * s.p.ny) == cudaSuccess;
            ok = ok && lb::launch_drive_profile(s.p.nx, s.p.ny, amp, s.d_drive, nullptr) == cudaSuccess;
        }
        if (ok && capped(s)) {
            ok = cudaMalloc(&s.d_umax, 2 * sizeof(double)) == cudaSuccess;
            if (ok) cudaMemset(s.d_umax, 0, 2 * sizeof(double));
        }
        ok = ok && cudaMalloc(&s.d_stats, kStatsAlloc) == cudaSuccess;
        if (ok) cudaMemset(s.d_stats, 0, kStatsAlloc);
        max_blocks = std::max<int64_t>(max_blocks, (s.N + lb::kDiagThreads - 1) / lb::kDiagThreads);
    }
    const size_t scratch = std::max<size_t>((size_t)max_blocks * lb::NPART, (size_t)lb::kMeansBlocks * lb::NMEANS);
    ok = ok && cudaMalloc(&h->d_scratch, scratch * sizeof(double)) == cudaSuccess;
    h->scratch_blocks = max_blocks;
    ok = ok && cudaMalloc(&h->d_small, 32 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->d_flag, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->d_status, sizeof(int)) == cudaSuccess;
    if (ok) cudaMemset(h->d_status, 0, sizeof(int));
    ok = ok && cudaMalloc(&h->d_barrier, 2 * sizeof(unsigned int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbrmhd_destroy(h);
        g_create_error = "device allocation failed";
        return LBRMHD_ERR_OOM;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        g_create_error = std::string("CUDA error during create: ") + cudaGetErrorString(cudaGetLastError());
        lbrmhd_destroy(h);
        return LBRMHD_ERR_CUDA;
    }
    for (size_t ri = 0; ri < h->runs.size(); ++ri) make_tile_maps(h->runs[ri], (int)ri);
    if (lookup_noalloc_scratch(&h->d_noalloc) != LBRMHD_OK) {
        g_create_error = "cudaGetSymbolAddress of the static diagnostics scratch failed";
        lbrmhd_destroy(h);
        return LBRMHD_ERR_CUDA;
    }
    *out = h;
    return LBRMHD_OK;
}

int lbrmhd_destroy(lbrmhd_handle h)
{
    if (!h) return LBRMHD_OK;
    cudaSetDevice(h->device);
    for (auto& r : h->runs) {
        for (int b = 0; b < 2; ++b) {
            if (r.pops[b]) cudaFree(r.pops[b]);
            if (r.h[b]) cudaFree(r.h[b]);
            if (r.prim[b]) cudaFree(r.prim[b]);
        }
        if (r.d_stats) cudaFree(r.d_stats);
        if (r.d_ez0) cudaFree(r.d_ez0);
        if (r.d_drive) cudaFree(r.d_drive);
        if (r.d_umax) cudaFree(r.d_umax);
        if (r.d_edge) cudaFree(r.d_edge);
    }
    if (h->d_scratch) cudaFree(h->d_scratch);
    if (h->d_io) cudaFree(h->d_io);
    if (h->d_small) cudaFree(h->d_small);
    if (h->d_flag) cudaFree(h->d_flag);
    if (h->d_status) cudaFree(h->d_status);
    if (h->d_barrier) cudaFree(h->d_barrier);
    if (h->d_mlp) cudaFree(h->d_mlp);
    drop_graphs(h);
    if (h->d_args) cudaFree(h->d_args);
    if (h->d_tiles) cudaFree(h->d_tiles);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    for (auto st : h->aux) cudaStreamDestroy(st);
    for (auto ev : h->aux_join) cudaEventDestroy(ev);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    delete h;
    return LBRMHD_OK;
}

int lbrmhd_set_stream(lbrmhd_handle h, void* stream)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    h->stream = (cudaStream_t)stream;
    return LBRMHD_OK;
}

int lbrmhd_init_fields(lbrmhd_handle h, int run, const double* n, const double* p, const double* u, const double* B,
                       const double* E)
{
    return init_common(h, run, n, p, u, B, E, false);
}

int lbrmhd_init_fields_relaxed(lbrmhd_handle h, int run, const double* n, const double* p, const double* u,
                               const double* B, int max_iters, double tol, int* iters, double* residual)
{
    if (bad_run(h, run)) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "run out of range") : LBRMHD_ERR_BAD_ARG;
    if (max_iters < 1 || !(tol >= 0)) return fail(h, LBRMHD_ERR_BAD_ARG, "max_iters must be >= 1 and tol >= 0");
    RunState& r = h->runs[run];
    if (r.p.bc[4] == LBRMHD_DRIVEN) return fail(h, LBRMHD_ERR_BAD_ARG, "relaxed initialisation of a DRIVEN run");
    int rc = init_common(h, run, n, p, u, B, nullptr, false);
    if (rc) return rc;
    switch (h->precision) {
        case LBRMHD_FP64: return relax_run<lb::CfgF64>(h, r, max_iters, tol, iters, residual);
        case LBRMHD_FP32: return relax_run<lb::CfgF32>(h, r, max_iters, tol, iters, residual);
        default: return relax_run<lb::CfgF16>(h, r, max_iters, tol, iters, residual);
    }
}

int lbrmhd_init_fields_device(lbrmhd_handle h, int run, const double* n, const double* p, const double* u,
                              const double* B, const double* E)
{
    return init_common(h, run, n, p, u, B, E, true);
}

int lbrmhd_step(lbrmhd_handle h, int64_t nsteps)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    if (nsteps < 0) return fail(h, LBRMHD_ERR_BAD_ARG, "nsteps < 0");
    for (auto& r : h->runs) {
        if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "lbrmhd_step before lbrmhd_init_fields");
        if (r.p.recovery == LBRMHD_RECOVERY_MLP && !h->mlp_set)
            return fail(h, LBRMHD_ERR_STATE, "learned-seed run without weights (lbrmhd_set_mlp_weights)");
    }
    for (auto& r : h->runs)
        if (r.cur != h->runs[0].cur) return fail(h, LBRMHD_ERR_STATE, "runs out of step");
    if (nsteps == 0) return LBRMHD_OK;
    LB_CK(cudaSetDevice(h->device));
    switch (h->precision) {
        case LBRMHD_FP64: return step_all<lb::CfgF64>(h, nsteps);
        case LBRMHD_FP32: return step_all<lb::CfgF32>(h, nsteps);
        default: return step_all<lb::CfgF16>(h, nsteps);
    }
}

int lbrmhd_get_moments_device(lbrmhd_handle h, int run, double* out)
{
    if (bad_run(h, run) || !out) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
    LB_CK(cudaSetDevice(h->device));
    const lb::Phys<double> k = make_phys<double>(r.p, r.ref, runref(r));
    switch (h->precision) {
        case LBRMHD_FP64: LB_CK(lb::launch_moments<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), k, out, h->stream)); break;
        case LBRMHD_FP32: LB_CK(lb::launch_moments<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), k, out, h->stream)); break;
        default: LB_CK(lb::launch_moments<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), k, out, h->stream)); break;
    }
    return LBRMHD_OK;
}

int lbrmhd_get_moments(lbrmhd_handle h, int run, double* out)
{
    if (bad_run(h, run) || !out) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    const int64_t N = h->runs[run].N;
    int rc = ensure_io(h, (size_t)LBRMHD_NMOMENTS * N * sizeof(double));
    if (rc) return rc;
    rc = lbrmhd_get_moments_device(h, run, h->d_io);
    if (rc) return rc;
    LB_CK(cudaMemcpyAsync(out, h->d_io, (size_t)LBRMHD_NMOMENTS * N * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

int lbrmhd_get_populations(lbrmhd_handle h, int run, double* f, double* g, double* hh)
{
    if (bad_run(h, run)) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "run out of range") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
    LB_CK(cudaSetDevice(h->device));
    const int64_t N = r.N;
    int rc = ensure_io(h, (size_t)63 * N * sizeof(double));
    if (rc) return rc;
    double* d = h->d_io;
    switch (h->precision) {
        case LBRMHD_FP64:
            LB_CK(lb::launch_populations<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), r.refpops, d, d + 19 * N, d + 38 * N,
                                                     h->stream));
            break;
        case LBRMHD_FP32:
            LB_CK(lb::launch_populations<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), r.refpops, d, d + 19 * N, d + 38 * N,
                                                     h->stream));
            break;
        default:
            LB_CK(lb::launch_populations<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), r.refpops, d, d + 19 * N, d + 38 * N,
                                                     h->stream));
            break;
    }
    if (f) LB_CK(cudaMemcpyAsync(f, d, 19 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (g) LB_CK(cudaMemcpyAsync(g, d + 19 * N, 19 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (hh) LB_CK(cudaMemcpyAsync(hh, d + 38 * N, 25 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

int lbrmhd_get_diagnostics(lbrmhd_handle h, int run, double* out)
{
    if (bad_run(h, run) || !out) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
    LB_CK(cudaSetDevice(h->device));
    const lb::Phys<double> k = make_phys<double>(r.p, r.ref, runref(r));
    switch (h->precision) {
        case LBRMHD_FP64:
            LB_CK(lb::launch_diag<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), k, r.ref, h->d_scratch, h->scratch_blocks,
                                              h->d_small, h->stream));
            break;
        case LBRMHD_FP32:
            LB_CK(lb::launch_diag<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), k, r.ref, h->d_scratch, h->scratch_blocks,
                                              h->d_small, h->stream));
            break;
        default:
            LB_CK(lb::launch_diag<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), k, r.ref, h->d_scratch, h->scratch_blocks,
                                              h->d_small, h->stream));
            break;
    }
    LB_CK(cudaMemcpyAsync(out, h->d_small, LBRMHD_NDIAG * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    if (out[8] > 0) return fail(h, LBRMHD_ERR_NONFINITE, "non-finite values in the state");
    return LBRMHD_OK;
}

int lbrmhd_get_diagnostics_noalloc(lbrmhd_handle h, int run, double* d_out)
{
    if (bad_run(h, run) || !d_out) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    if (r.N > kNoAllocMaxCells)
        return fail(h, LBRMHD_ERR_BAD_ARG,
                    "lbrmhd_get_diagnostics_noalloc: run has " + std::to_string(r.N) + " cells, above the limit of " +
                        std::to_string(kNoAllocMaxCells) + " of its static scratch; use lbrmhd_get_diagnostics");
    if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
    LB_CK(cudaSetDevice(h->device));
    double* partial = h->d_noalloc;
    const lb::Phys<double> k = make_phys<double>(r.p, r.ref, runref(r));
    switch (h->precision) {
        case LBRMHD_FP64:
            LB_CK(lb::launch_diag<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), k, r.ref, partial, kNoAllocMaxBlocks, d_out,
                                              h->stream));
            break;
        case LBRMHD_FP32:
            LB_CK(lb::launch_diag<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), k, r.ref, partial, kNoAllocMaxBlocks, d_out,
                                              h->stream));
            break;
        default:
            LB_CK(lb::launch_diag<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), k, r.ref, partial, kNoAllocMaxBlocks, d_out,
                                              h->stream));
            break;
    }
    return LBRMHD_OK;
}

int lbrmhd_barrier_selftest(lbrmhd_handle h, int unreachable, double wait_seconds)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    if (!(wait_seconds > 0.0 && wait_seconds <= 10.0)) return fail(h, LBRMHD_ERR_BAD_ARG, "wait_seconds must be in (0, 10]");
    LB_CK(cudaSetDevice(h->device));
    // scratch: d_small's first 8 bytes as counter + status (not the handle's status word)
    unsigned int* counter = reinterpret_cast<unsigned int*>(h->d_small);
    int* status = reinterpret_cast<int*>(h->d_small) + 1;
    LB_CK(cudaMemsetAsync(h->d_small, 0, 2 * sizeof(int), h->stream));
    int dev_sms = 0;
    LB_CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device));
    LB_CK(lb::launch_barrier_selftest(std::min(dev_sms, 8), counter, status, unreachable,
                                      (unsigned long long)(wait_seconds * 1e9), h->stream));
    int st = 0;
    LB_CK(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    if (st & lb::STATUS_BARRIER_TIMEOUT) return fail(h, LBRMHD_ERR_TIMEOUT, "grid barrier wait ran out");
    return LBRMHD_OK;
}

int lbrmhd_get_status(lbrmhd_handle h, int64_t* out3)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    LB_CK(cudaSetDevice(h->device));
    int status = 0;
    LB_CK(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    int64_t fails = 0, tiled = 0;
    const bool per_run = effective_schedule(h).kind == LBRMHD_SCHED_PER_RUN;  // the tile kernel's only schedule
    for (const auto& r : h->runs) {
        unsigned long long s[lb::kNumStats];
        const int rc = read_stats(h, r, s);
        if (rc) return rc;
        fails += (int64_t)s[0];
        tiled += per_run && !r.tmaps.empty() && (r.p.flags & LBRMHD_FLAG_TMA_TILES) != 0 &&
                         (r.p.flags & LBRMHD_FLAG_GAUSS_CHARGE) == 0
                     ? 1
                     : 0;
    }
    if (out3) {
        out3[0] = status;
        out3[1] = fails;
        out3[2] = tiled;
    }
    if (status & lb::STATUS_TMA_TIMEOUT) return fail(h, LBRMHD_ERR_TIMEOUT, "a TMA tile copy did not arrive in time");
    if (status & lb::STATUS_BARRIER_TIMEOUT) return fail(h, LBRMHD_ERR_TIMEOUT, "a grid barrier wait ran out");
    if (fails > 0) return fail(h, LBRMHD_ERR_NONCONVERGED, std::to_string(fails) + " recoveries did not converge");
    return LBRMHD_OK;
}

int lbrmhd_get_stats(lbrmhd_handle h, int run, int64_t* out4)
{
    if (bad_run(h, run) || !out4) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    LB_CK(cudaSetDevice(h->device));
    unsigned long long s[lb::kNumStats];
    const int rc = read_stats(h, r, s);
    if (rc) return rc;
    out4[0] = r.steps;
    out4[1] = (int64_t)s[0];
    out4[2] = (int64_t)s[1];
    out4[3] = (int64_t)s[2];
    return LBRMHD_OK;
}

int lbrmhd_get_iteration_histogram(lbrmhd_handle h, int run, int64_t* out)
{
    if (bad_run(h, run) || !out) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    LB_CK(cudaSetDevice(h->device));
    unsigned long long s[lb::kNumStats];
    const int rc = read_stats(h, r, s);
    if (rc) return rc;
    for (int b = 0; b < lb::kHistBins; ++b) out[b] = (int64_t)s[3 + b];
    return LBRMHD_OK;
}

// checkpoint blob: [uint64 layout tag] then per run [int64 steps][NMEANS double
// reference means][uint64 stats x kNumStats][pops 38 N][h 25 N][prim 12 N]
// [initial E^z N] (storage format). The tag names the storage layout (fluid
// groups as 4-vectors, Maxwell pairs as 2-vectors, primitive 4-vectors) and the
// precision; a blob of another layout is refused.
constexpr uint64_t kStateLayoutTag = 0x4c42524d48440200ull;  // "LBRMHD", layout 2, low byte = precision
uint64_t state_tag(int precision) { return kStateLayoutTag | (uint64_t)(precision & 0xff); }

int lbrmhd_state_bytes(lbrmhd_handle h, size_t* bytes)
{
    if (!h || !bytes) return LBRMHD_ERR_BAD_ARG;
    const size_t pb = pop_bytes(h->precision), hb = hp_bytes(h->precision);
    size_t total = 8;
    for (auto& r : h->runs)
        total += 8 + 8 * lb::NMEANS + kStatsBytes + (size_t)r.N * (38 * pb + 25 * hb + (lb::NPRIM + 1) * hb);
    *bytes = total;
    return LBRMHD_OK;
}

int lbrmhd_get_state(lbrmhd_handle h, void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (lbrmhd_state_bytes(h, &need) || !host_buf || bytes != need)
        return h ? fail(h, LBRMHD_ERR_BAD_ARG, "state buffer size mismatch") : LBRMHD_ERR_BAD_ARG;
    LB_CK(cudaSetDevice(h->device));
    const size_t pb = pop_bytes(h->precision), hb = hp_bytes(h->precision);
    char* o = (char*)host_buf;
    const uint64_t tag = state_tag(h->precision);
    std::memcpy(o, &tag, 8);
    o += 8;
    for (auto& r : h->runs) {
        if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
        std::memcpy(o, &r.steps, 8);
        o += 8;
        std::memcpy(o, r.means, 8 * lb::NMEANS);
        o += 8 * lb::NMEANS;
        unsigned long long tot[lb::kNumStats];
        const int rc = read_stats(h, r, tot);
        if (rc) return rc;
        std::memcpy(o, tot, kStatsBytes);
        o += kStatsBytes;
        for (const Segment& sg : state_segments(r, true)) {
            LB_CK(cudaMemcpyAsync(o, (char*)r.pops[r.cur] + sg.first * pb, sg.count * pb, cudaMemcpyDeviceToHost,
                                  h->stream));
            o += sg.count * pb;
        }
        for (const Segment& sg : state_segments(r, false)) {
            LB_CK(cudaMemcpyAsync(o, (char*)r.h[r.cur] + sg.first * hb, sg.count * hb, cudaMemcpyDeviceToHost,
                                  h->stream));
            o += sg.count * hb;
        }
        for (int q = 0; q < lb::kPrimVecs; ++q, o += 4 * r.N * hb)
            LB_CK(cudaMemcpyAsync(o, (char*)r.prim[r.cur] + lb::prim_elem(4 * q, 0, r.stride) * hb, 4 * r.N * hb,
                                  cudaMemcpyDeviceToHost, h->stream));
        LB_CK(cudaMemcpyAsync(o, r.d_ez0, r.N * hb, cudaMemcpyDeviceToHost, h->stream));
        o += r.N * hb;
    }
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

int lbrmhd_set_state(lbrmhd_handle h, const void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (lbrmhd_state_bytes(h, &need) || !host_buf || bytes != need)
        return h ? fail(h, LBRMHD_ERR_BAD_ARG, "state buffer size mismatch") : LBRMHD_ERR_BAD_ARG;
    LB_CK(cudaSetDevice(h->device));
    const size_t pb = pop_bytes(h->precision), hb = hp_bytes(h->precision);
    const char* o = (const char*)host_buf;
    uint64_t tag = 0;
    std::memcpy(&tag, o, 8);
    if (tag != state_tag(h->precision))
        return fail(h, LBRMHD_ERR_BAD_ARG, "checkpoint of another storage layout or precision");
    o += 8;
    for (auto& r : h->runs) {
        std::memcpy(&r.steps, o, 8);
        o += 8;
        double means[lb::NMEANS];
        std::memcpy(means, o, 8 * lb::NMEANS);
        o += 8 * lb::NMEANS;
        set_reference(r, means);
        unsigned long long tot[lb::kNumStats];
        std::memcpy(tot, o, kStatsBytes);
        const int rc = write_stats(h, r, tot);
        if (rc) return rc;
        o += kStatsBytes;
        for (const Segment& sg : state_segments(r, true)) {
            LB_CK(cudaMemcpyAsync((char*)r.pops[r.cur] + sg.first * pb, o, sg.count * pb, cudaMemcpyHostToDevice,
                                  h->stream));
            o += sg.count * pb;
        }
        for (const Segment& sg : state_segments(r, false)) {
            LB_CK(cudaMemcpyAsync((char*)r.h[r.cur] + sg.first * hb, o, sg.count * hb, cudaMemcpyHostToDevice,
                                  h->stream));
            o += sg.count * hb;
        }
        for (int q = 0; q < lb::kPrimVecs; ++q, o += 4 * r.N * hb)
            LB_CK(cudaMemcpyAsync((char*)r.prim[r.cur] + lb::prim_elem(4 * q, 0, r.stride) * hb, o, 4 * r.N * hb,
                                  cudaMemcpyHostToDevice, h->stream));
        LB_CK(cudaMemcpyAsync(r.d_ez0, o, r.N * hb, cudaMemcpyHostToDevice, h->stream));
        o += r.N * hb;
        const int rc2 = refresh_umax(h, r);
        if (rc2) return rc2;
        r.initialized = true;
        runs_changed(h);
    }
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

int64_t lbrmhd_run_cells(lbrmhd_handle h, int run)
{
    if (bad_run(h, run)) return 0;
    return h->runs[run].N;
}

int lbrmhd_set_mlp_weights(lbrmhd_handle h, const float* d_params)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    if (!d_params) return fail(h, LBRMHD_ERR_BAD_ARG, "NULL parameters");
    LB_CK(cudaSetDevice(h->device));
    if (!h->d_mlp && cudaMalloc(&h->d_mlp, lbrmhd_mlp_blob_bytes()) != cudaSuccess) {
        h->d_mlp = nullptr;
        return fail(h, LBRMHD_ERR_OOM, "network blob allocation failed");
    }
    const int rc = lbrmhd_mlp_pack(d_params, h->d_mlp, h->stream);
    if (rc) return fail(h, rc, "packing the network failed");
    h->mlp_set = true;
    runs_changed(h);  // the kernel arguments carry the blob pointer
    return LBRMHD_OK;
}

int lbrmhd_set_mlp_samples(lbrmhd_handle h, int run, float* d_samples)
{
    if (bad_run(h, run)) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "run out of range") : LBRMHD_ERR_BAD_ARG;
    h->runs[run].d_samples = d_samples;
    runs_changed(h);
    return LBRMHD_OK;
}

int lbrmhd_set_schedule(lbrmhd_handle h, const lbrmhd_schedule* sched)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    if (!sched) return fail(h, LBRMHD_ERR_BAD_ARG, "NULL schedule");
    const std::string m = check_schedule(*sched);
    if (!m.empty()) return fail(h, LBRMHD_ERR_BAD_ARG, m);
    h->sched = *sched;
    h->tiles_dirty = true;
    drop_graphs(h);
    return LBRMHD_OK;
}

int lbrmhd_get_schedule(lbrmhd_handle h, lbrmhd_schedule* sched)
{
    if (!h || !sched) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "NULL schedule") : LBRMHD_ERR_BAD_ARG;
    *sched = effective_schedule(h);
    return LBRMHD_OK;
}

int lbrmhd_autotune(lbrmhd_handle h, int trials, lbrmhd_schedule* best, double* best_ms)
{
    if (!h) return LBRMHD_ERR_BAD_ARG;
    if (trials < 1 || trials > 100) return fail(h, LBRMHD_ERR_BAD_ARG, "trials must be in 1..100");
    LB_CK(cudaSetDevice(h->device));
    switch (h->precision) {
        case LBRMHD_FP64: return autotune<lb::CfgF64>(h, trials, best, best_ms);
        case LBRMHD_FP32: return autotune<lb::CfgF32>(h, trials, best, best_ms);
        default: return autotune<lb::CfgF16>(h, trials, best, best_ms);
    }
}

int lbrmhd_reconnection_rate(lbrmhd_handle h, int run, int y_lo, int y_hi, double B0, double* out4)
{
    if (bad_run(h, run) || !out4) return h ? fail(h, LBRMHD_ERR_BAD_ARG, "bad run or NULL output") : LBRMHD_ERR_BAD_ARG;
    RunState& r = h->runs[run];
    if (r.p.nz != 1) return fail(h, LBRMHD_ERR_BAD_ARG, "the reconnection rate is defined for 2-D runs");
    if (y_lo < 0 || y_hi > r.p.ny || y_lo >= y_hi) return fail(h, LBRMHD_ERR_BAD_ARG, "empty or out-of-grid row band");
    if (!(B0 != 0.0) || !std::isfinite(B0)) return fail(h, LBRMHD_ERR_BAD_ARG, "B0 must be finite and non-zero");
    if (!r.initialized) return fail(h, LBRMHD_ERR_STATE, "run not initialised");
    LB_CK(cudaSetDevice(h->device));
    const int64_t scratch = std::max<int64_t>(h->scratch_blocks * lb::NPART, (int64_t)lb::kMeansBlocks * lb::NMEANS);
    cudaError_t e;
    switch (h->precision) {
        case LBRMHD_FP64:
            e = lb::launch_null<lb::CfgF64>(view<lb::CfgF64>(r, r.cur), y_lo, y_hi, (const double*)r.d_ez0, B0,
                                            h->d_scratch, scratch, h->d_small, h->stream);
            break;
        case LBRMHD_FP32:
            e = lb::launch_null<lb::CfgF32>(view<lb::CfgF32>(r, r.cur), y_lo, y_hi, (const float*)r.d_ez0, B0,
                                            h->d_scratch, scratch, h->d_small, h->stream);
            break;
        default:
            e = lb::launch_null<lb::CfgF16>(view<lb::CfgF16>(r, r.cur), y_lo, y_hi, (const float*)r.d_ez0, B0,
                                            h->d_scratch, scratch, h->d_small, h->stream);
            break;
    }
    LB_CK(e);
    LB_CK(cudaMemcpyAsync(out4, h->d_small, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB_CK(cudaStreamSynchronize(h->stream));
    return LBRMHD_OK;
}

const char* lbrmhd_last_error(lbrmhd_handle h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int lbrmhd_lattice_tables(double* out, size_t n)
{
    if (!out || n < LBRMHD_NTABLE) return LBRMHD_ERR_BAD_ARG;
    double* o = out;
    for (int i = 0; i < 19; ++i)
        for (int a = 0; a < 3; ++a) *o++ = lb::c19(i, a);
    for (int i = 0; i < 19; ++i) *o++ = lb::w19(i);
    for (int i = 0; i < 19; ++i) *o++ = lb::wg19(i);
    for (int k = 0; k < 24; ++k)
        for (int a = 0; a < 3; ++a) *o++ = lb::hop13(k, a);
    for (int k = 0; k < 24; ++k) {  // e_k / c
        const int p = k / 8, i = (k % 8) / 2, j = k % 2, ie = (i + 3) % 4;
        const double s = (j == 0 ? 1.0 : -1.0) * lb::kSqrt2 / 2.0;
        for (int a = 0; a < 3; ++a)
            *o++ = a == lb::plane_a1(p) ? s * lb::hop_s1(ie) : (a == lb::plane_a2(p) ? s * lb::hop_s2(ie) : 0.0);
    }
    for (int k = 0; k < 24; ++k) {  // b_k
        const int p = k / 8, j = k % 2;
        for (int a = 0; a < 3; ++a)
            *o++ = a == lb::plane_normal(p) ? (j == 0 ? -1.0 : 1.0) * lb::plane_orient(p) : 0.0;
    }
    return LBRMHD_OK;
}

}  // extern "C"
