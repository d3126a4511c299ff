// Host side of liblcdm: argument checks, workspace carving, launch shapes,
// the launch-shape autotuner, and the extern "C" entry points of include/lcdm.h.
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/lcdm.h"
#include "lcdm_between.cuh"
#include "lcdm_launch.cuh"
#include "lcdm_prep.cuh"
#include "lcdm_redshift.cuh"

using namespace lcdm;

namespace {

std::atomic<int64_t> g_launches{0};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// largest batch whose root preparation uses four lanes per cosmology
#define LCDM_PREP_GROUP_MAX_B 16384

size_t ws_bytes_for(int64_t B) {
    return align256((size_t)B * NREC * sizeof(double)) + align256((size_t)B * NREC * sizeof(float2));
}

bool opts_ok(const lcdm_opts* o) {
    return o && (o->ncol == 4 || o->ncol == 5 || o->ncol == 7) &&
           (o->precision == LCDM_FP64 || o->precision == LCDM_FP32_MIXED) &&
           o->layout >= LCDM_LAYOUT_CSR && o->layout <= LCDM_LAYOUT_SHARED && o->block >= 0 && o->block <= 256 &&
           (o->block % 32) == 0 && o->blocks_per_sm >= 0 && o->blocks_per_sm <= 64 && o->lane_map >= LCDM_MAP_TUNED &&
           o->lane_map <= LCDM_MAP_INTERLEAVED && (o->deterministic == 0 || o->deterministic == 1);
}

int num_sms();

// Partial sums of the deterministic reduction: per launched warp, the sums
// of its first and last rows (DET_NV values each) and those rows' indices.
// At most 64 resident warps per SM are ever launched.
#define DET_NV (RF_KT + 2)
size_t det_warps() { return (size_t)64 * num_sms(); }
size_t det_bytes() {
    return align256(det_warps() * 2 * DET_NV * sizeof(double)) + align256(det_warps() * 2 * sizeof(int64_t));
}

struct Carved {
    double* recD;
    float2* recF;
    double* part = nullptr;      // deterministic mode: [warps][2][DET_NV]
    int64_t* wrow = nullptr;     // [warps][2]
};

lcdm_status carve(void* ws, size_t ws_bytes, int64_t B, Carved& c, int det = 0) {
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < ws_bytes_for(B) + (det ? det_bytes() : 0))
        return LCDM_ERR_WORKSPACE;
    c.recD = (double*)ws;
    c.recF = (float2*)((char*)ws + align256((size_t)B * NREC * sizeof(double)));
    if (det) {
        c.part = (double*)((char*)ws + ws_bytes_for(B));
        c.wrow = (int64_t*)((char*)c.part + align256(det_warps() * 2 * DET_NV * sizeof(double)));
    }
    return LCDM_OK;
}

// SM count of the current device, looked up once per device
#define LCDM_MAX_DEVICES 64
std::atomic<int> g_num_sms[LCDM_MAX_DEVICES];

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LCDM_MAX_DEVICES) dev = 0;
    return dev;
}

int num_sms() {
    const int dev = current_device();
    int n = g_num_sms[dev].load();
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_num_sms[dev].store(n);
    }
    return n;
}

const PairsTable& table(int prec, int K) {
    static PairsTable t[2][4];
    static std::once_flag once;
    std::call_once(once, [] {
        t[0][0] = table_f64_k0(); t[0][1] = table_f64_k3(); t[0][2] = table_f64_k4(); t[0][3] = table_f64_k6();
        t[1][0] = table_mix_k0(); t[1][1] = table_mix_k3(); t[1][2] = table_mix_k4(); t[1][3] = table_mix_k6();
    });
    return t[prec][K == 0 ? 0 : (K == 3 ? 1 : (K == 4 ? 2 : 3))];
}

// tuned launch shapes: key (device, precision, K, WT, WX, layout, log2 npairs)
typedef std::tuple<int, int, int, int, int, int, int> TuneKey;
struct Tuned { int block, bps, lane_map; };
std::map<TuneKey, Tuned> g_tuned;
std::mutex g_tune_mu;

int log2_bucket(int64_t n) {
    int b = 0;
    while (n > 1) { n >>= 1; b++; }
    return b;
}

struct Plan {
    PairArgs args;
    int prec, K, wt, wx;
    int64_t npairs;
    TuneKey key;
    // outputs wanted as values only while other outputs need tangents: the
    // time coordinate and the absorption distance each run their own R_J
    // track, whose tangents would be computed for nothing; such outputs are
    // written by a second, tangent-free launch (split_mask: LCDM_T, LCDM_X bits)
    int split_mask;
};

lcdm_status check_pairs_args(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                             int32_t* status, const lcdm_opts* opts) {
    if (!opts_ok(opts) || !params || !status || B <= 0 || n < 0) return LCDM_ERR_INVALID;
    if (opts->layout == LCDM_LAYOUT_CSR && !offsets) return LCDM_ERR_INVALID;
    if (n > 0 && !z) return LCDM_ERR_INVALID;
    return LCDM_OK;
}

// Builds the kernel arguments; any of out / jac / cot / mobs may be null.
lcdm_status make_plan(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                      void* const* out, void* const* jac, const void* const* cot, const void* mobs, double M,
                      double sigma, double* grad, double* loglike, int32_t* status, const lcdm_opts* opts,
                      const Carved& cv, Plan& P) {
    PairArgs& a = P.args;
    memset(&a, 0, sizeof(a));
    a.recD = cv.recD;
    a.recF = cv.recF;
    a.part = cv.part;
    a.wrow = cv.wrow;
    a.det_cap = cv.part ? (int64_t)det_warps() : 0;
    a.status = status;
    a.offsets = offsets;
    a.z = z;
    a.layout = opts->layout;
    a.B = B;
    a.ncol = opts->ncol;
    a.nrow = n;
    P.npairs = opts->layout == LCDM_LAYOUT_CSR ? n : B * n;
    a.nnz = P.npairs;
    bool tangents = grad != nullptr;
    int wt = 0, wx = 0;
    for (int i = 0; i < LCDM_NOUT; i++) {
        a.out[i] = out ? out[i] : nullptr;
        a.jac[i] = jac ? jac[i] : nullptr;
        a.cot[i] = cot ? cot[i] : nullptr;
        if (a.out[i]) a.outmask |= 1 << i;
        if (a.jac[i]) tangents = true;
        bool used = a.out[i] || a.jac[i] || a.cot[i];
        if (used && i == LCDM_T) wt = 1;
        if (used && i == LCDM_X) wx = 1;
    }
    P.split_mask = 0;
    if (mobs) { tangents = tangents || grad != nullptr; }
    a.mobs = mobs;
    a.M = M;
    a.sigma = sigma;
    a.grad = grad;
    a.loglike = loglike;
    P.prec = opts->precision == LCDM_FP64 ? 0 : 1;
    P.K = tangents ? opts->ncol - 1 : 0;
    if (P.K > 0) {
        for (int i : {LCDM_T, LCDM_X}) {
            if (a.out[i] && !a.jac[i] && !a.cot[i]) {
                P.split_mask |= 1 << i;
                if (i == LCDM_T) wt = 0;
                if (i == LCDM_X) wx = 0;
            }
        }
    }
    P.wt = wt;
    P.wx = wx;
    P.key = TuneKey(current_device(), P.prec, P.K, wt, wx, opts->layout, log2_bucket(P.npairs));
    return LCDM_OK;
}

lcdm_status launch_one(Plan& P, int block, int bps, int lane_map, cudaStream_t s);

}  // namespace

namespace lcdm {
// The deterministic reduction's second pass: the shared rows' partial sums
// added in warp order by one thread (a few thousand additions).
__global__ void det_fixup_kernel(PairArgs a, int64_t nwarps) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int64_t w = 0; w < nwarps && w < a.det_cap; w++) {
        for (int k = 0; k < 2; k++) {
            const int64_t r = a.wrow[w * 2 + k];
            if (r < 0 || (k == 1 && r == a.wrow[w * 2])) continue;
            const double* v = a.part + (w * 2 + k) * DET_SLOT;
            if (a.grad) for (int i = 0; i < a.ncol; i++) a.grad[r * a.ncol + i] += v[i];
            if (a.loglike) a.loglike[r] += v[DET_SLOT - 1];
        }
    }
}

cudaError_t launch_det_fixup(const PairArgs& a, int64_t nwarps, cudaStream_t s) {
    det_fixup_kernel<<<1, 32, 0, s>>>(a, nwarps);
    return cudaGetLastError();
}
}  // namespace lcdm

namespace {

// The plan's launches: the value-only outputs of split_mask first (K = 0,
// their tracks only, no reductions), then the tangent launch without them.
lcdm_status launch_plan(Plan& P, int block, int bps, int lane_map, cudaStream_t s) {
    if (P.split_mask) {
        Plan V = P;
        PairArgs& v = V.args;
        v.outmask = 0;
        for (int i = 0; i < LCDM_NOUT; i++) {
            v.jac[i] = nullptr;
            v.cot[i] = nullptr;
            if (!(P.split_mask & (1 << i))) v.out[i] = nullptr;
            if (v.out[i]) v.outmask |= 1 << i;
        }
        v.mobs = nullptr;
        v.grad = nullptr;
        v.loglike = nullptr;
        V.K = 0;
        V.wt = (P.split_mask >> LCDM_T) & 1;
        V.wx = (P.split_mask >> LCDM_X) & 1;
        V.split_mask = 0;
        std::get<2>(V.key) = 0;
        std::get<3>(V.key) = V.wt;
        std::get<4>(V.key) = V.wx;
        lcdm_status st = launch_one(V, 0, 0, lane_map, s);
        if (st != LCDM_OK) return st;
        Plan T = P;
        for (int i = 0; i < LCDM_NOUT; i++)
            if (P.split_mask & (1 << i)) { T.args.out[i] = nullptr; T.args.outmask &= ~(1 << i); }
        T.split_mask = 0;
        return launch_one(T, block, bps, lane_map, s);
    }
    return launch_one(P, block, bps, lane_map, s);
}

// Resident blocks per SM of a pair kernel, queried once per (device, kernel,
// block size): the query is host work on every launch otherwise (the chunked
// host entry point launches twice per chunk).
int cached_occ(const PairsTable& t, int idx, int prec, int K, int block) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int>, int> cache;
    const auto key = std::make_tuple(current_device(), prec, K, idx, block);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int occ = t.occ[idx](block);
    if (occ > 0) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = occ;
    }
    return occ;
}
lcdm_status launch_one(Plan& P, int block, int bps, int lane_map, cudaStream_t s) {
    const PairsTable& t = table(P.prec, P.K);
    int idx = (P.wt ? 2 : 0) + (P.wx ? 1 : 0);
    if (block == 0 || bps == 0 || lane_map == LCDM_MAP_TUNED) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(P.key);
        if (it != g_tuned.end()) {
            if (block == 0) block = it->second.block;
            if (bps == 0) bps = it->second.bps;
            if (lane_map == LCDM_MAP_TUNED) lane_map = it->second.lane_map;
        }
    }
    P.args.interleave = lane_map == LCDM_MAP_INTERLEAVED ? 1 : 0;
    if (block == 0) block = 256;   // full-size blocks (the largest kernels step in lockstep, see pairs_kernel)
    int occ = cached_occ(t, idx, P.prec, P.K, block);
    if (occ <= 0) return LCDM_ERR_CUDA;
    if (bps == 0 || bps > occ) bps = occ;
    int64_t warps = (int64_t)num_sms() * bps * (block / 32);
    int64_t chunk = (P.npairs + warps - 1) / warps;
    chunk = ((chunk + 31) / 32) * 32;
    if (chunk < 32) chunk = 32;
    P.args.chunk = chunk;
    int64_t need_warps = (P.npairs + chunk - 1) / chunk;
    int64_t grid = (need_warps * 32 + block - 1) / block;
    if (grid < 1) grid = 1;
    if (P.npairs == 0) return LCDM_OK;
    cudaError_t e = t.launch[idx](P.args, (int)grid, block, s);
    g_launches++;
    if (e != cudaSuccess) return LCDM_ERR_CUDA;
    if (P.args.part && (P.args.grad || P.args.loglike)) {
        // the shared rows' partial sums, added in warp order
        e = launch_det_fixup(P.args, need_warps, s);
        g_launches++;
    }
    return e == cudaSuccess ? LCDM_OK : LCDM_ERR_CUDA;
}

lcdm_status run_prep(const double* params, int64_t B, const lcdm_opts* opts, const Carved& cv, int32_t* status,
                     double* grad, double* loglike, cudaStream_t s) {
    // One warp per block, so that the FP64 work spreads over as many SMs as
    // possible.  Up to LCDM_PREP_GROUP_MAX_B cosmologies the solve is bound by
    // the latency of one cosmology's dependent FP64 chain and four lanes share
    // each root solve; beyond that the FP64 pipe is the bound and one lane per
    // cosmology does no repeated work.
    const int block = 32;
    if (B <= LCDM_PREP_GROUP_MAX_B) {
        const int64_t grid = (4 * B + block - 1) / block;
        prep_kernel<4><<<(unsigned)grid, block, 0, s>>>(params, B, opts->ncol, cv.recD, cv.recF, status, grad,
                                                       loglike);
    } else {
        const int64_t grid = (B + block - 1) / block;
        prep_kernel<1><<<(unsigned)grid, block, 0, s>>>(params, B, opts->ncol, cv.recD, cv.recF, status, grad,
                                                       loglike);
    }
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? LCDM_OK : LCDM_ERR_CUDA;
}

__global__ void extract_roots(const double* __restrict__ recD, int64_t B, int ncol, double* roots, double* droots,
                              int32_t* kind) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* r = recD + b * NREC;
    int kd = (int)r[RF_KIND];
    bool cpair = kd == 0 || kd == 2, quartic = kd <= 1;
    int K = ncol - 1;
    if (kind) kind[b] = kd;
    // slots: A, B, pair member 1, pair member 2
    double re[4] = {r[RF_A], quartic ? r[RF_B] : -0.0, r[RF_PRE], cpair ? r[RF_PRE] : r[RF_PIM]};
    double im[4] = {0, 0, cpair ? r[RF_PIM] : 0.0, cpair ? -r[RF_PIM] : 0.0};
    if (roots)
        for (int s = 0; s < 4; s++) { roots[(b * 4 + s) * 2] = re[s]; roots[(b * 4 + s) * 2 + 1] = im[s]; }
    if (droots) {
        for (int k = 0; k < K; k++) {
            double dre[4] = {r[RF_DA + k], quartic ? r[RF_DB + k] : 0.0, r[RF_DPRE + k],
                             cpair ? r[RF_DPRE + k] : r[RF_DPIM + k]};
            double dim[4] = {0, 0, cpair ? r[RF_DPIM + k] : 0.0, cpair ? -r[RF_DPIM + k] : 0.0};
            for (int s = 0; s < 4; s++) {
                droots[((b * 4 + s) * 2 + 0) * K + k] = dre[s];
                droots[((b * 4 + s) * 2 + 1) * K + k] = dim[s];
            }
        }
    }
}

lcdm_status pairs_common(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                         void* const* out, void* const* jac, const void* const* cot, const void* mobs, double M,
                         double sigma, double* grad, double* loglike, int32_t* status, const lcdm_opts* opts,
                         void* ws, size_t ws_bytes, cudaStream_t stream) {
    lcdm_status st = check_pairs_args(params, B, offsets, z, n, status, opts);
    if (st != LCDM_OK) return st;
    Carved cv;
    st = carve(ws, ws_bytes, B, cv, opts->deterministic);
    if (st != LCDM_OK) return st;
    Plan P;
    st = make_plan(params, B, offsets, z, n, out, jac, cot, mobs, M, sigma, grad, loglike, status, opts, cv, P);
    if (st != LCDM_OK) return st;
    st = run_prep(params, B, opts, cv, status, grad, loglike, stream);
    if (st != LCDM_OK) return st;
    return launch_plan(P, opts->block, opts->blocks_per_sm, opts->lane_map, stream);
}

// ----------------------------------------------------------------------------
// Fixed device scratch for lcdm_distances_static.  The array belongs to this
// translation unit; its device address is looked up once per device with
// cudaGetSymbolAddress (the host-side name is only a stand-in and must never
// be handed to a kernel).
// ----------------------------------------------------------------------------
#define LCDM_STATIC_WS_BYTES (((size_t)LCDM_STATIC_MAX_COSMOLOGIES * NREC * sizeof(double) + 255) / 256 * 256 + \
                              ((size_t)LCDM_STATIC_MAX_COSMOLOGIES * NREC * sizeof(float2) + 255) / 256 * 256)
static __device__ __align__(256) unsigned char g_static_ws[LCDM_STATIC_WS_BYTES];

static void* g_static_ptr[LCDM_MAX_DEVICES];
static std::mutex g_static_mu;

// Device address of g_static_ws on the current device (set up on first use).
static lcdm_status static_workspace(void** ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LCDM_MAX_DEVICES) return LCDM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return LCDM_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *ptr = g_static_ptr[dev];
    return LCDM_OK;
}

// ----------------------------------------------------------------------------
// Host-buffer entry point: chunked copies on two internal streams per device
// (host-to-device and device-to-host) overlapping the pair kernel of the
// neighbouring chunks on the caller's stream.
// ----------------------------------------------------------------------------
#define LCDM_HOST_MAX_CHUNKS 64
struct HostStreams {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev[2 * LCDM_HOST_MAX_CHUNKS + 3];
    bool ready = false;
};
static HostStreams g_host_streams[LCDM_MAX_DEVICES];
static std::mutex g_host_mu;

lcdm_status host_streams(HostStreams** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LCDM_MAX_DEVICES) return LCDM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_host_mu);
    HostStreams& h = g_host_streams[dev];
    if (!h.ready) {
        if (cudaStreamCreateWithFlags(&h.up, cudaStreamNonBlocking) != cudaSuccess) return LCDM_ERR_CUDA;
        if (cudaStreamCreateWithFlags(&h.down, cudaStreamNonBlocking) != cudaSuccess) return LCDM_ERR_CUDA;
        for (int i = 0; i < 2 * LCDM_HOST_MAX_CHUNKS + 3; i++)
            if (cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming) != cudaSuccess) return LCDM_ERR_CUDA;
        h.ready = true;
    }
    *out = &h;
    return LCDM_OK;
}

// Device workspace of the host entry point: records, then params, offsets,
// status, grad, z, six cotangent and six output arrays.
struct HostCarve {
    Carved rec;
    double* params;
    int64_t* offsets;
    int32_t* status;
    double* grad;
    char* z;
    char* cot[LCDM_NOUT];
    char* out[LCDM_NOUT];
    size_t bytes;
};

HostCarve host_carve(char* base, int64_t B, int64_t n, int ncol, size_t es) {
    HostCarve c;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
    char* rec = take(ws_bytes_for(B));
    c.rec.recD = (double*)rec;
    c.rec.recF = rec ? (float2*)(rec + align256((size_t)B * NREC * sizeof(double))) : nullptr;
    c.params = (double*)take((size_t)B * ncol * sizeof(double));
    c.offsets = (int64_t*)take((size_t)(B + 1) * sizeof(int64_t));
    c.status = (int32_t*)take((size_t)B * sizeof(int32_t));
    c.grad = (double*)take((size_t)B * ncol * sizeof(double));
    c.z = take((size_t)n * es);
    for (int i = 0; i < LCDM_NOUT; i++) c.cot[i] = take((size_t)n * es);
    for (int i = 0; i < LCDM_NOUT; i++) c.out[i] = take((size_t)n * es);
    c.bytes = off;
    return c;
}

// Device workspace of the general-limits entry points: records of the
// shifted cosmologies, shifted parameters (closure form, four columns), their
// Jacobian, the scale s = 1+z1,
// the gradient w.r.t. the shifted parameters, z' and three scaled cotangents
// (d_C, X, d_M).
struct BetweenCarve {
    Carved rec;
    double* params4;
    double* jac;
    double* scale;
    float4* rowf;
    double* gradp;
    char* zp;
    char* cotp[LCDM_NOUT];
    size_t bytes;
};

BetweenCarve between_carve(char* base, int64_t B, int64_t npairs, int ncol, size_t es) {
    BetweenCarve c;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
    char* rec = take(ws_bytes_for(B));
    c.rec.recD = (double*)rec;
    c.rec.recF = rec ? (float2*)(rec + align256((size_t)B * NREC * sizeof(double))) : nullptr;
    c.params4 = (double*)take((size_t)B * 4 * sizeof(double));
    c.jac = (double*)take((size_t)B * 4 * ncol * sizeof(double));
    c.scale = (double*)take((size_t)B * sizeof(double));
    c.rowf = (float4*)take((size_t)B * sizeof(float4));
    c.gradp = (double*)take((size_t)B * 4 * sizeof(double));
    c.zp = take((size_t)npairs * es);
    for (int i = 0; i < LCDM_NOUT; i++) c.cotp[i] = nullptr;
    c.cotp[LCDM_DC] = take((size_t)npairs * es);
    c.cotp[LCDM_X] = take((size_t)npairs * es);
    c.cotp[LCDM_DM] = take((size_t)npairs * es);
    c.bytes = off;
    return c;
}

lcdm_status between_npairs(int64_t B, int64_t n, const lcdm_opts* opts, int64_t* npairs) {
    if (!opts_ok(opts) || B <= 0 || n < 0 || (n > 0 && opts->layout == LCDM_LAYOUT_SHARED))
        return LCDM_ERR_INVALID;
    *npairs = opts->layout == LCDM_LAYOUT_CSR ? n : B * n;
    return LCDM_OK;
}

// Shift every row to its lower limit and prepare the shifted records.
lcdm_status between_setup(const double* params, int64_t B, const double* z1, int ncol, const BetweenCarve& w,
                          const lcdm_opts* opts4, int32_t* status, double* gradp, cudaStream_t stream) {
    ShiftArgs sa;
    sa.params = params;
    sa.z1 = z1;
    sa.B = B;
    sa.ncol = ncol;
    sa.params4 = w.params4;
    sa.jac = w.jac;
    sa.scale = w.scale;
    sa.rowf = w.rowf;
    if (launch_shift(sa, stream) != cudaSuccess) return LCDM_ERR_CUDA;
    g_launches++;
    return run_prep(w.params4, B, opts4, w.rec, status, gradp, nullptr, stream);
}

}  // namespace

extern "C" {

lcdm_status lcdm_between_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes) {
    int64_t npairs = 0;
    if (!bytes || between_npairs(B, n, opts, &npairs) != LCDM_OK) return LCDM_ERR_INVALID;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    *bytes = between_carve(nullptr, B, npairs, opts->ncol, es).bytes;
    return LCDM_OK;
}

lcdm_status lcdm_distances_between(const double* params, int64_t B, const double* z1, const int64_t* offsets,
                                   const void* z2, int64_t n, const void* const cot[LCDM_NOUT],
                                   void* const out[LCDM_NOUT], double* grad, int32_t* cosmo_status,
                                   const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
    int64_t npairs = 0;
    if (between_npairs(B, n, opts, &npairs) != LCDM_OK || !z1 || (!out && !grad) || (grad && !cot))
        return LCDM_ERR_INVALID;
    if (opts->ncol > 5) return LCDM_ERR_UNSUPPORTED;   // the row shift takes 4 or 5 columns
    if (opts->deterministic && grad) return LCDM_ERR_UNSUPPORTED;
    lcdm_status st = check_pairs_args(params, B, offsets, z2, n, cosmo_status, opts);
    if (st != LCDM_OK) return st;
    const int ncol = opts->ncol;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    if (!ws || ((uintptr_t)ws & 255) != 0) return LCDM_ERR_WORKSPACE;
    BetweenCarve w = between_carve((char*)ws, B, npairs, ncol, es);
    if (ws_bytes < w.bytes) return LCDM_ERR_WORKSPACE;
    lcdm_opts o4 = *opts;
    o4.ncol = 4;
    st = between_setup(params, B, z1, ncol, w, &o4, cosmo_status, grad ? w.gradp : nullptr, stream);
    if (st != LCDM_OK) return st;
    PairMapArgs m;
    memset(&m, 0, sizeof(m));
    m.offsets = opts->layout == LCDM_LAYOUT_CSR ? offsets : nullptr;
    m.nrow = n;
    m.nnz = npairs;
    m.B = B;
    m.fp64 = opts->precision == LCDM_FP64;
    m.z1 = z1;
    m.scale = w.scale;
    m.rowf = w.rowf;
    m.z2 = z2;
    m.zp = w.zp;
    const void* cotk[LCDM_NOUT] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (grad)
        for (int i = 0; i < LCDM_NOUT; i++) {
            m.cot[i] = cot[i];
            cotk[i] = cot[i];
            if (cot[i] && w.cotp[i]) { m.cotp[i] = w.cotp[i]; cotk[i] = w.cotp[i]; }
        }
    if (launch_pair_pre(m, stream) != cudaSuccess) return LCDM_ERR_CUDA;
    g_launches++;
    Plan P;
    make_plan(w.params4, B, offsets, w.zp, n, out, nullptr, grad ? cotk : nullptr, nullptr, 0, 1,
              grad ? w.gradp : nullptr, nullptr, cosmo_status, &o4, w.rec, P);
    st = launch_plan(P, opts->block, opts->blocks_per_sm, opts->lane_map, stream);
    if (st != LCDM_OK) return st;
    if (out) {
        for (int i = 0; i < LCDM_NOUT; i++) m.out[i] = out[i];
        if (launch_pair_post(m, stream) != cudaSuccess) return LCDM_ERR_CUDA;
        g_launches++;
    }
    if (grad) {
        if (launch_chain(w.jac, w.gradp, B, ncol, grad, stream) != cudaSuccess) return LCDM_ERR_CUDA;
        g_launches++;
    }
    return LCDM_OK;
}

lcdm_status lcdm_loglike_dz_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes) {
    if (!opts_ok(opts) || B <= 0 || n < 0 || !bytes) return LCDM_ERR_INVALID;
    const int64_t npairs = opts->layout == LCDM_LAYOUT_CSR ? n : B * n;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    *bytes = align256(ws_bytes_for(B)) + 2 * align256((size_t)npairs * es);
    return LCDM_OK;
}

lcdm_status lcdm_gauss_loglike_dz(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  const void* m_obs, int64_t n, double M, double sigma, double* loglike,
                                  double* grad, void* grad_z, void* mu_out, int32_t* cosmo_status,
                                  const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!m_obs || !loglike || !grad_z || !(sigma > 0) || !std::isfinite(M)) return LCDM_ERR_INVALID;
    lcdm_status st = check_pairs_args(params, B, offsets, z, n, cosmo_status, opts);
    if (st != LCDM_OK) return st;
    if (opts->ncol > 5) return LCDM_ERR_UNSUPPORTED;   // E(z) of the redshift kernel: 4 or 5 columns
    if (opts->deterministic) return LCDM_ERR_UNSUPPORTED;
    size_t need = 0;
    lcdm_loglike_dz_workspace_size(B, n, opts, &need);
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < need) return LCDM_ERR_WORKSPACE;
    const int64_t npairs = opts->layout == LCDM_LAYOUT_CSR ? n : B * n;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    Carved cv;
    carve(ws, ws_bytes, B, cv);
    char* dC = (char*)ws + align256(ws_bytes_for(B));
    char* mu = dC + align256((size_t)npairs * es);
    if (mu_out) mu = (char*)mu_out;
    void* out[LCDM_NOUT] = {dC, nullptr, nullptr, nullptr, nullptr, mu};
    Plan P;
    st = make_plan(params, B, offsets, z, n, out, nullptr, nullptr, m_obs, M, sigma, grad, loglike, cosmo_status,
                   opts, cv, P);
    if (st != LCDM_OK) return st;
    st = run_prep(params, B, opts, cv, cosmo_status, grad, loglike, stream);
    if (st != LCDM_OK) return st;
    st = launch_plan(P, opts->block, opts->blocks_per_sm, opts->lane_map, stream);
    if (st != LCDM_OK) return st;
    DzArgs d;
    d.params = params;
    d.ncol = opts->ncol;
    d.status = cosmo_status;
    d.offsets = offsets;
    d.layout = opts->layout;
    d.nrow = n;
    d.nnz = npairs;
    d.B = B;
    d.fp64 = opts->precision == LCDM_FP64;
    d.z = z;
    d.mobs = m_obs;
    d.dC = dC;
    d.mu = mu;
    d.M = M;
    d.sigma = sigma;
    for (int i = 0; i < LCDM_NOUT; i++) d.cot[i] = nullptr;
    d.vjp = 0;
    d.grad_z = grad_z;
    if (launch_loglike_dz(d, stream) != cudaSuccess) return LCDM_ERR_CUDA;
    g_launches++;
    return LCDM_OK;
}

lcdm_status lcdm_distances_vjp_dz(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  int64_t n, const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT],
                                  double* grad, void* grad_z, int32_t* cosmo_status, const lcdm_opts* opts,
                                  void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!cot || !grad_z) return LCDM_ERR_INVALID;
    lcdm_status st = check_pairs_args(params, B, offsets, z, n, cosmo_status, opts);
    if (st != LCDM_OK) return st;
    if (opts->ncol > 5) return LCDM_ERR_UNSUPPORTED;   // E(z) of the redshift kernel: 4 or 5 columns
    if (opts->deterministic && grad) return LCDM_ERR_UNSUPPORTED;
    size_t need = 0;
    lcdm_loglike_dz_workspace_size(B, n, opts, &need);
    if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < need) return LCDM_ERR_WORKSPACE;
    const int64_t npairs = opts->layout == LCDM_LAYOUT_CSR ? n : B * n;
    Carved cv;
    carve(ws, ws_bytes, B, cv);
    void* outk[LCDM_NOUT];
    for (int i = 0; i < LCDM_NOUT; i++) outk[i] = out ? out[i] : nullptr;
    if (!outk[LCDM_DC]) outk[LCDM_DC] = (char*)ws + align256(ws_bytes_for(B));   // d_C feeds the z-derivatives
    Plan P;
    st = make_plan(params, B, offsets, z, n, outk, nullptr, grad ? cot : nullptr, nullptr, 0, 1, grad, nullptr,
                   cosmo_status, opts, cv, P);
    if (st != LCDM_OK) return st;
    st = run_prep(params, B, opts, cv, cosmo_status, grad, nullptr, stream);
    if (st != LCDM_OK) return st;
    st = launch_plan(P, opts->block, opts->blocks_per_sm, opts->lane_map, stream);
    if (st != LCDM_OK) return st;
    DzArgs d;
    memset(&d, 0, sizeof(d));
    d.params = params;
    d.ncol = opts->ncol;
    d.status = cosmo_status;
    d.offsets = offsets;
    d.layout = opts->layout;
    d.nrow = n;
    d.nnz = npairs;
    d.B = B;
    d.fp64 = opts->precision == LCDM_FP64;
    d.z = z;
    d.dC = outk[LCDM_DC];
    d.sigma = 1.0;
    for (int i = 0; i < LCDM_NOUT; i++) d.cot[i] = cot[i];
    d.vjp = 1;
    d.grad_z = grad_z;
    if (launch_loglike_dz(d, stream) != cudaSuccess) return LCDM_ERR_CUDA;
    g_launches++;
    return LCDM_OK;
}

lcdm_status lcdm_limits(const double* params, int64_t B, const double* z1, double* chi_inf, double* t_inf,
                        const double* cot_chi, const double* cot_t, double* grad, int32_t* cosmo_status,
                        const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!opts_ok(opts) || B <= 0 || !params || !z1 || !cosmo_status || (!chi_inf && !t_inf && !grad))
        return LCDM_ERR_INVALID;
    if (opts->ncol > 5) return LCDM_ERR_UNSUPPORTED;   // the row shift takes 4 or 5 columns
    const int ncol = opts->ncol;
    if (!ws || ((uintptr_t)ws & 255) != 0) return LCDM_ERR_WORKSPACE;
    BetweenCarve w = between_carve((char*)ws, B, 0, ncol, 8);
    if (ws_bytes < w.bytes) return LCDM_ERR_WORKSPACE;
    lcdm_opts o4 = *opts;
    o4.ncol = 4;
    lcdm_status st = between_setup(params, B, z1, ncol, w, &o4, cosmo_status, nullptr, stream);
    if (st != LCDM_OK) return st;
    LimitArgs la;
    la.recD = w.rec.recD;
    la.recF = w.rec.recF;
    la.status = cosmo_status;
    la.B = B;
    la.scale = w.scale;
    la.chi = chi_inf;
    la.age = t_inf;
    la.cot_chi = cot_chi;
    la.cot_age = cot_t;
    la.gradp = w.gradp;
    if (launch_limits(la, grad != nullptr, stream) != cudaSuccess) return LCDM_ERR_CUDA;
    g_launches++;
    if (grad) {
        if (launch_chain(w.jac, w.gradp, B, ncol, grad, stream) != cudaSuccess) return LCDM_ERR_CUDA;
        g_launches++;
    }
    return LCDM_OK;
}

lcdm_status lcdm_distances_static(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                  int64_t n, void* const out[LCDM_NOUT], int32_t* cosmo_status,
                                  const lcdm_opts* opts, cudaStream_t stream) {
    if (!out || B > LCDM_STATIC_MAX_COSMOLOGIES) return LCDM_ERR_INVALID;
    lcdm_status st = check_pairs_args(params, B, offsets, z, n, cosmo_status, opts);
    if (st != LCDM_OK) return st;
    void* ws = nullptr;
    st = static_workspace(&ws);
    if (st != LCDM_OK) return st;
    lcdm_opts o = *opts;
    o.deterministic = 0;   // forward values only: there is no reduction
    return pairs_common(params, B, offsets, z, n, out, nullptr, nullptr, nullptr, 0, 1, nullptr, nullptr,
                        cosmo_status, &o, ws, LCDM_STATIC_WS_BYTES, stream);
}


lcdm_status lcdm_host_workspace_size(int64_t B, int64_t n, const lcdm_opts* opts, size_t* bytes) {
    if (!opts_ok(opts) || B <= 0 || n < 0 || !bytes) return LCDM_ERR_INVALID;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    *bytes = host_carve(nullptr, B, n, opts->ncol, es).bytes;
    return LCDM_OK;
}

lcdm_status lcdm_distances_vjp_host(const double* params, int64_t B, const int64_t* offsets, const void* z,
                                    int64_t n, const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT],
                                    double* grad, int32_t* cosmo_status, const lcdm_opts* opts, void* dws,
                                    size_t dws_bytes, int32_t nchunks, cudaStream_t stream) {
    if (!opts_ok(opts) || opts->layout != LCDM_LAYOUT_CSR || !params || !offsets || B <= 0 || n < 0 ||
        (n > 0 && !z) || !cot || !grad || !cosmo_status || nchunks < 1 || nchunks > LCDM_HOST_MAX_CHUNKS)
        return LCDM_ERR_INVALID;
    if (offsets[0] != 0 || offsets[B] != n) return LCDM_ERR_INVALID;
    if (opts->deterministic) return LCDM_ERR_UNSUPPORTED;
    for (int64_t r = 0; r < B; r++)
        if (offsets[r + 1] < offsets[r]) return LCDM_ERR_INVALID;
    const int ncol = opts->ncol;
    const size_t es = opts->precision == LCDM_FP64 ? 8 : 4;
    if (!dws || ((uintptr_t)dws & 255) != 0) return LCDM_ERR_WORKSPACE;
    HostCarve d = host_carve((char*)dws, B, n, ncol, es);
    if (dws_bytes < d.bytes) return LCDM_ERR_WORKSPACE;
    HostStreams* hs = nullptr;
    lcdm_status st = host_streams(&hs);
    if (st != LCDM_OK) return st;
    cudaEvent_t* ev = hs->ev;
    bool ok = true;
    auto chk = [&](cudaError_t e) { ok = ok && e == cudaSuccess; };
    // the copies wait for earlier work on the caller's stream (workspace reuse)
    chk(cudaEventRecord(ev[0], stream));
    chk(cudaStreamWaitEvent(hs->up, ev[0], 0));
    chk(cudaMemcpyAsync(d.params, params, (size_t)B * ncol * sizeof(double), cudaMemcpyHostToDevice, hs->up));
    chk(cudaMemcpyAsync(d.offsets, offsets, (size_t)(B + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, hs->up));
    chk(cudaEventRecord(ev[1], hs->up));
    chk(cudaStreamWaitEvent(stream, ev[1], 0));
    if (!ok) return LCDM_ERR_CUDA;
    st = run_prep(d.params, B, opts, d.rec, d.status, d.grad, nullptr, stream);
    if (st != LCDM_OK) return st;
    // chunk c covers rows [rb[c], rb[c+1]); its share of the pairs ramps up and
    // down, weights min(c + 1, nchunks - c, 3) (1 2 3 ... 3 2 1): the first
    // chunk's input copy and the last chunk's output copy are the parts of the
    // pipeline that nothing overlaps, and each step of the ramp at most doubles
    // (or halves) a chunk, so the next chunk's copy still hides behind the
    // current chunk's kernels
    int64_t rb[LCDM_HOST_MAX_CHUNKS + 1];
    int64_t wcum[LCDM_HOST_MAX_CHUNKS + 1];
    wcum[0] = 0;
    for (int c = 0; c < nchunks; c++) {
        int w = c + 1 < nchunks - c ? c + 1 : nchunks - c;
        wcum[c + 1] = wcum[c] + (w < 3 ? w : 3);
    }
    rb[0] = 0;
    for (int c = 1; c < nchunks; c++) {
        const int64_t target = (int64_t)((double)n * (double)wcum[c] / (double)wcum[nchunks]);
        int64_t lo = rb[c - 1], hi = B;   // first row whose start offset is >= target
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (offsets[mid] < target) lo = mid + 1; else hi = mid;
        }
        rb[c] = lo;
    }
    rb[nchunks] = B;
    for (int c = 0; c < nchunks; c++) {
        const int64_t r0 = rb[c], r1 = rb[c + 1];
        const int64_t o0 = offsets[r0], o1 = offsets[r1];
        if (r1 <= r0 || o1 <= o0) continue;
        const size_t nb = (size_t)(o1 - o0) * es, ob = (size_t)o0 * es;
        chk(cudaMemcpyAsync(d.z + ob, (const char*)z + ob, nb, cudaMemcpyHostToDevice, hs->up));
        const void* cotd[LCDM_NOUT] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        void* outd[LCDM_NOUT] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        for (int i = 0; i < LCDM_NOUT; i++) {
            if (cot[i]) {
                chk(cudaMemcpyAsync(d.cot[i] + ob, (const char*)cot[i] + ob, nb, cudaMemcpyHostToDevice, hs->up));
                cotd[i] = d.cot[i];
            }
            if (out && out[i]) outd[i] = d.out[i];
        }
        chk(cudaEventRecord(ev[2 + 2 * c], hs->up));
        chk(cudaStreamWaitEvent(stream, ev[2 + 2 * c], 0));
        if (!ok) return LCDM_ERR_CUDA;
        Carved rc;
        rc.recD = d.rec.recD + r0 * NREC;
        rc.recF = d.rec.recF + r0 * NREC;
        Plan P;
        make_plan(d.params + r0 * ncol, r1 - r0, d.offsets + r0, d.z, o1 - o0, outd, nullptr, cotd, nullptr, 0, 1,
                  d.grad + r0 * ncol, nullptr, d.status + r0, opts, rc, P);
        P.args.base = o0;
        st = launch_plan(P, opts->block, opts->blocks_per_sm, opts->lane_map, stream);
        if (st != LCDM_OK) return st;
        chk(cudaEventRecord(ev[3 + 2 * c], stream));
        chk(cudaStreamWaitEvent(hs->down, ev[3 + 2 * c], 0));
        for (int i = 0; i < LCDM_NOUT; i++)
            if (outd[i]) chk(cudaMemcpyAsync((char*)out[i] + ob, d.out[i] + ob, nb, cudaMemcpyDeviceToHost, hs->down));
        if (!ok) return LCDM_ERR_CUDA;
    }
    chk(cudaEventRecord(ev[2 * LCDM_HOST_MAX_CHUNKS + 2], stream));
    chk(cudaStreamWaitEvent(hs->down, ev[2 * LCDM_HOST_MAX_CHUNKS + 2], 0));
    chk(cudaMemcpyAsync(grad, d.grad, (size_t)B * ncol * sizeof(double), cudaMemcpyDeviceToHost, hs->down));
    chk(cudaMemcpyAsync(cosmo_status, d.status, (size_t)B * sizeof(int32_t), cudaMemcpyDeviceToHost, hs->down));
    chk(cudaStreamSynchronize(hs->down));
    return ok ? LCDM_OK : LCDM_ERR_CUDA;
}

lcdm_status lcdm_workspace_size(int64_t B, const lcdm_opts* opts, size_t* bytes) {
    if (!opts_ok(opts) || B <= 0 || !bytes) return LCDM_ERR_INVALID;
    *bytes = ws_bytes_for(B) + (opts->deterministic ? det_bytes() : 0);
    return LCDM_OK;
}

lcdm_status lcdm_roots(const double* params, int64_t B, const lcdm_opts* opts, double* roots, double* droots,
                       int32_t* kind, int32_t* cosmo_status, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!opts_ok(opts) || !params || !cosmo_status || B <= 0) return LCDM_ERR_INVALID;
    Carved cv;
    lcdm_status st = carve(ws, ws_bytes, B, cv);
    if (st != LCDM_OK) return st;
    st = run_prep(params, B, opts, cv, cosmo_status, nullptr, nullptr, stream);
    if (st != LCDM_OK) return st;
    extract_roots<<<(unsigned)((B + 127) / 128), 128, 0, stream>>>(cv.recD, B, opts->ncol, roots, droots, kind);
    g_launches++;
    return cudaGetLastError() == cudaSuccess ? LCDM_OK : LCDM_ERR_CUDA;
}

lcdm_status lcdm_distances(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                           void* const out[LCDM_NOUT], int32_t* cosmo_status, const lcdm_opts* opts, void* ws,
                           size_t ws_bytes, cudaStream_t stream) {
    if (!out) return LCDM_ERR_INVALID;
    return pairs_common(params, B, offsets, z, n, out, nullptr, nullptr, nullptr, 0, 1, nullptr, nullptr,
                        cosmo_status, opts, ws, ws_bytes, stream);
}

lcdm_status lcdm_distances_jac(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                               void* const out[LCDM_NOUT], void* const jac[LCDM_NOUT], int32_t* cosmo_status,
                               const lcdm_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!jac) return LCDM_ERR_INVALID;
    return pairs_common(params, B, offsets, z, n, out, jac, nullptr, nullptr, 0, 1, nullptr, nullptr,
                        cosmo_status, opts, ws, ws_bytes, stream);
}

lcdm_status lcdm_distances_vjp(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                               const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT], double* grad,
                               int32_t* cosmo_status, const lcdm_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream) {
    if (!cot || !grad) return LCDM_ERR_INVALID;
    return pairs_common(params, B, offsets, z, n, out, nullptr, cot, nullptr, 0, 1, grad, nullptr, cosmo_status,
                        opts, ws, ws_bytes, stream);
}

lcdm_status lcdm_gauss_loglike(const double* params, int64_t B, const int64_t* offsets, const void* z,
                               const void* m_obs, int64_t n, double M, double sigma, double* loglike, double* grad,
                               void* mu_out, int32_t* cosmo_status, const lcdm_opts* opts, void* ws,
                               size_t ws_bytes, cudaStream_t stream) {
    if (!m_obs || !loglike || !(sigma > 0) || !std::isfinite(M)) return LCDM_ERR_INVALID;
    void* out[LCDM_NOUT] = {nullptr, nullptr, nullptr, nullptr, nullptr, mu_out};
    return pairs_common(params, B, offsets, z, n, out, nullptr, nullptr, m_obs, M, sigma, grad, loglike,
                        cosmo_status, opts, ws, ws_bytes, stream);
}

lcdm_status lcdm_autotune(const double* params, int64_t B, const int64_t* offsets, const void* z, int64_t n,
                          const void* const cot[LCDM_NOUT], void* const out[LCDM_NOUT], double* grad,
                          int32_t* cosmo_status, const lcdm_opts* opts, void* ws, size_t ws_bytes,
                          cudaStream_t stream, int32_t* best_block, int32_t* best_bps, float* best_ms,
                          int32_t* best_map) {
    lcdm_status st = check_pairs_args(params, B, offsets, z, n, cosmo_status, opts);
    if (st != LCDM_OK) return st;
    if (!grad) cot = nullptr;   // forward-only shape
    Carved cv;
    st = carve(ws, ws_bytes, B, cv, opts->deterministic);
    if (st != LCDM_OK) return st;
    Plan P;
    st = make_plan(params, B, offsets, z, n, out, nullptr, cot, nullptr, 0, 1, grad, nullptr, cosmo_status, opts, cv,
                   P);
    if (st != LCDM_OK) return st;
    const PairsTable& t = table(P.prec, P.K);
    int idx = (P.wt ? 2 : 0) + (P.wx ? 1 : 0);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LCDM_ERR_CUDA;
    const int blocks[] = {64, 128, 256};
    float best = 1e30f;
    int bb = 128, bbps = 1, bmap = LCDM_MAP_CONTIGUOUS;
    for (int map = LCDM_MAP_CONTIGUOUS; map <= LCDM_MAP_INTERLEAVED; map++) {
        if (opts->lane_map != LCDM_MAP_TUNED && map != opts->lane_map) continue;
        for (int block : blocks) {
            int occ = t.occ[idx](block);
            for (int bps = 1; bps <= occ; bps = (bps * 2 > occ && bps < occ) ? occ : bps * 2) {
                float tot = 0;
                for (int rep = 0; rep < 3; rep++) {
                    if (run_prep(params, B, opts, cv, cosmo_status, grad, nullptr, stream) != LCDM_OK)
                        return LCDM_ERR_CUDA;
                    cudaEventRecord(e0, stream);
                    if (launch_plan(P, block, bps, map, stream) != LCDM_OK) return LCDM_ERR_CUDA;
                    cudaEventRecord(e1, stream);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tot += ms;
                }
                tot /= 2;
                if (tot < best) { best = tot; bb = block; bbps = bps; bmap = map; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[P.key] = Tuned{bb, bbps, bmap};
    }
    if (best_block) *best_block = bb;
    if (best_bps) *best_bps = bbps;
    if (best_ms) *best_ms = best;
    if (best_map) *best_map = bmap;
    return cudaGetLastError() == cudaSuccess ? LCDM_OK : LCDM_ERR_CUDA;
}

const char* lcdm_status_string(int s) {
    switch (s) {
        case LCDM_OK: return "LCDM_OK";
        case LCDM_ERR_INVALID: return "LCDM_ERR_INVALID: invalid argument";
        case LCDM_ERR_CUDA: return "LCDM_ERR_CUDA: CUDA launch or query failed";
        case LCDM_ERR_WORKSPACE: return "LCDM_ERR_WORKSPACE: workspace missing, too small or not 256-byte aligned";
        case LCDM_ERR_UNSUPPORTED: return "LCDM_ERR_UNSUPPORTED: unsupported combination";
        default: return "unknown lcdm_status";
    }
}

int64_t lcdm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
