// lbm_capi.cu -- the C ABI of include/lbm.h: contexts, device memory layout,
// TMA tensor maps, parameters, launches (optionally from CUDA graphs),
// read-back, checkpoints, the tile/schedule autotuner and the host-side EOS
// helpers (critical point, Maxwell coexistence, Laplace fit).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm_eos_host.h"
#include "lbm_init.h"
#include "lbm_internal.cuh"

using lbm::Inst;

namespace {

constexpr unsigned long long kTimeoutNs = 1000000000ull;   // bounded TMA wait: 1 s
#ifndef LBM_RUN_CHUNK_MB
#define LBM_RUN_CHUNK_MB 80   // populations per multi-step launch, MiB (see build_run_chunks)
#endif

// An NVTX range over the enclosing scope (host side: it brackets the calls
// that enqueue or wait for the work); a no-op unless a profiler is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};
constexpr int kGraphLevels = 5;                            // captured graphs of 2, 4, ..., 32 steps
constexpr int kGraphSteps = 2 << (kGraphLevels - 1);       // the longest: 32 steps
constexpr int kReadBands = 8;                              // row bands of a field read-back
constexpr size_t kReadBandMin = size_t(1) << 20;           // nodes from which the read-back is banded

// The TMA tensor maps of one instance's two time levels (host copies; the
// kernels receive them in their argument blocks).
struct Maps {
    CUtensorMap tmap[2];
};

struct HostParams {
    lbm_eos eos;
    double A, kappa, G, s[9], rho_ref;
    unsigned flags;
    int set;
    int var_visc;
    double nu_g, nu_l, visc_rho_g, visc_rho_l;
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int esize(int prec) { return prec == LBM_FP32 ? 4 : (prec == LBM_FP64 ? 8 : 0); }
int ghost_x(int prec) { return prec == LBM_FP32 ? lbm::Prec<float>::GX : lbm::Prec<double>::GX; }

int pitch_of(int nx, int prec) {
    const int per32 = 32 / esize(prec);
    return static_cast<int>(align_up(static_cast<size_t>(ghost_x(prec) + nx + 2), per32));
}

struct Layout {
    std::vector<size_t> pop_off[2];
    size_t inst_off, tiles_off, status_off, partials_off, result_off, scratch_off, run_off, total;
    size_t tiles_cap, scratch_elems;
};

bool valid_shape(int n, const int* nx, const int* ny, int prec) {
    if (n < 1 || !nx || !ny || esize(prec) == 0) return false;
    for (int i = 0; i < n; ++i)
        if (nx[i] < 2 || ny[i] < 2 || nx[i] > (1 << 20) || ny[i] > (1 << 20)) return false;
    return true;
}

Layout make_layout(int n, const int* nx, const int* ny, int prec) {
    Layout L;
    size_t off = 0;
    const size_t es = esize(prec);
    size_t maxN = 0, tiles = 0;
    for (int i = 0; i < n; ++i) {
        const size_t plane = static_cast<size_t>(pitch_of(nx[i], prec)) * (ny[i] + 2 * lbm::GY);
        for (int k = 0; k < 2; ++k) {
            L.pop_off[k].push_back(off);
            off = align_up(off + 9 * plane * es, 256);
        }
        maxN = std::max(maxN, static_cast<size_t>(nx[i]) * ny[i]);
    }
    for (int c = 0; c < lbm::step_config_count(prec); ++c) {
        const lbm::TileCfg t = lbm::step_config(prec, c);
        size_t s = 0;
        for (int i = 0; i < n; ++i) s += static_cast<size_t>((nx[i] + t.bx - 1) / t.bx) * ((ny[i] + t.by - 1) / t.by);
        tiles = std::max(tiles, s);
    }
    L.inst_off = off;
    off = align_up(off + n * sizeof(Inst), 256);
    L.tiles_off = off;
    L.tiles_cap = tiles;
    off = align_up(off + tiles * sizeof(int4), 256);
    L.status_off = off;
    off = align_up(off + n * sizeof(int), 256);
    L.partials_off = off;
    off = align_up(off + lbm::kReduceBlocks * lbm::kReduceSlots * sizeof(double), 256);
    L.result_off = off;
    off = align_up(off + lbm::kReduceSlots * sizeof(double), 256);
    L.scratch_off = off;
    L.scratch_elems = 3 * maxN;
    off = align_up(off + L.scratch_elems * sizeof(double), 256);
    L.run_off = off;   // multi-step launches: work counter, abort flag, then one step counter per tile
    off = align_up(off + 16 + tiles * sizeof(int), 256);
    L.total = off;
    return L;
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// ---- host EOS (independent numerical routines) ---------------------------
double eos_p(const lbm_eos& e, double rho) {
    const double RT = e.R * e.T;
    if (e.kind == LBM_EOS_CS) {
        const double n = e.b * rho / 4.0, q = 1.0 - n;
        return e.K * (rho * RT * (1.0 + n + n * n - n * n * n) / (q * q * q) - e.a * rho * rho);
    }
    if (e.kind == LBM_EOS_VDW) return e.K * (rho * RT / (1.0 - e.b * rho) - e.a * rho * rho);
    const double br = e.b * rho;
    return e.K * (rho * RT / (1.0 - br) - e.a * lbm::pr_alpha(e) * rho * rho / (1.0 + 2.0 * br - br * br));
}

double eos_dp(const lbm_eos& e, double rho) {
    const double RT = e.R * e.T;
    if (e.kind == LBM_EOS_CS) {
        const double n = e.b * rho / 4.0, q = 1.0 - n;
        return e.K * (RT * (1.0 + 4.0 * n + 4.0 * n * n - 4.0 * n * n * n + n * n * n * n) / (q * q * q * q) -
                      2.0 * e.a * rho);
    }
    if (e.kind == LBM_EOS_VDW) {
        const double q = 1.0 - e.b * rho;
        return e.K * (RT / (q * q) - 2.0 * e.a * rho);
    }
    const double br = e.b * rho, D = 1.0 + 2.0 * br - br * br, q = 1.0 - br;
    return e.K * (RT / (q * q) - e.a * lbm::pr_alpha(e) * (2.0 * rho + 2.0 * e.b * rho * rho) / (D * D));
}

double eos_rho_max(const lbm_eos& e) { return e.kind == LBM_EOS_CS ? 4.0 / e.b : 1.0 / e.b; }

using lbm::eos_valid;

// argmin over (lo, hi) of a unimodal function, golden section
template <class F> double golden_min(F f, double lo, double hi, double* fmin) {
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double a = lo, b = hi, c = b - g * (b - a), d = a + g * (b - a);
    double fc = f(c), fd = f(d);
    for (int it = 0; it < 300 && (b - a) > 1e-15 * (std::fabs(a) + std::fabs(b)); ++it) {
        if (fc < fd) { b = d; d = c; fd = fc; c = b - g * (b - a); fc = f(c); }
        else { a = c; c = d; fc = fd; d = a + g * (b - a); fd = f(d); }
    }
    const double x = 0.5 * (a + b);
    *fmin = f(x);
    return x;
}

template <class F> double bisect(F f, double lo, double hi) {
    double flo = f(lo);
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return 0.5 * (lo + hi);
}

// composite 8-point Gauss-Legendre
double gauss_int(const lbm_eos& e, double p0, double a, double b, int panels) {
    static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    double s = 0.0;
    const double h = (b - a) / panels;
    for (int k = 0; k < panels; ++k) {
        const double c = a + (k + 0.5) * h, r = 0.5 * h;
        for (int j = 0; j < 4; ++j)
            for (int sg = -1; sg <= 1; sg += 2) {
                const double x = c + sg * r * xg[j];
                s += wg[j] * r * (p0 - eos_p(e, x)) / (x * x);
            }
    }
    return s;
}

}  // namespace

struct lbm_ctx {
    int n = 0, prec = 0, esz = 0, device = 0;
    std::vector<int> nx, ny;
    std::vector<Inst> h;
    std::vector<HostParams> hp;
    std::vector<int> inited;
    Layout L;
    char* buf = nullptr;
    size_t buf_bytes = 0;
    bool owns = false;
    cudaStream_t stream = nullptr;
    Inst* d_inst = nullptr;
    int4* d_tiles = nullptr;
    int ntiles = 0;                   // tiles of all instances
    std::vector<Maps> maps;
    // a batch (n > 1) is stepped by one launch per chunk of up to
    // kBatchLaunchMax instances: argument blocks per time-level parity
    std::vector<lbm::BatchArgs<float>> bargs_f[2];
    std::vector<lbm::BatchArgs<double>> bargs_d[2];
    std::vector<int> chunk_tiles;
    // schedule 3 (multi-step persistent launches): one argument block per chunk
    // of up to kRunMax instances, and each chunk's first tile in the step counters
    std::vector<lbm::RunArgs<float>> rargs_f;
    std::vector<lbm::RunArgs<double>> rargs_d;
    std::vector<int> run_first;
    char* d_run = nullptr;
    int* d_status = nullptr;
    double* d_partials = nullptr;
    double* d_result = nullptr;
    double* d_scratch = nullptr;
    int parity = 0;
    long long steps = 0, launches = 0;
    int cfg = 0, sched = 0;
    bool use_graphs = false;
    cudaGraphExec_t gexec[2][kGraphLevels] = {};   // [start parity][level]: 2 << level steps
    lbm::StepArgs<float> one_f{};    // kernel argument block of a one-lattice context
    lbm::StepArgs<double> one_d{};
    // field read-back of a large lattice: row bands computed on `stream`
    // while the bands before them are copied to the host on copy_stream
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t band_done[kReadBands] = {};
    std::string err;
};

namespace {

int fail(lbm_ctx* c, int code, const char* fmt, const char* detail = "") {
    if (c) {
        char b[512];
        std::snprintf(b, sizeof b, fmt, detail);
        c->err = b;
    }
    return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_ECUDA;
}

#define CK(c, call)                                            \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
    } while (0)

void drop_graphs(lbm_ctx* c) {
    for (auto& per : c->gexec)
        for (auto& g : per)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int encode_maps(lbm_ctx* c) {
    EncodeTiled enc = get_encoder();
    if (!enc) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver%s");
    const lbm::TileCfg t = lbm::step_config(c->prec, c->cfg);
    const int HX = c->prec == LBM_FP32 ? lbm::Prec<float>::HX : lbm::Prec<double>::HX;
    for (int i = 0; i < c->n; ++i) {
        Inst& I = c->h[i];
        for (int k = 0; k < 2; ++k) {
            cuuint64_t dims[3] = {static_cast<cuuint64_t>(I.pitch), static_cast<cuuint64_t>(I.nyp), 9};
            cuuint64_t strides[2] = {static_cast<cuuint64_t>(I.pitch) * c->esz,
                                     static_cast<cuuint64_t>(I.plane) * c->esz};
            cuuint32_t box[3] = {static_cast<cuuint32_t>(t.bx + 2 * HX), static_cast<cuuint32_t>(t.by + 2 * lbm::GY), 9};
            cuuint32_t es[3] = {1, 1, 1};
            CUresult r = enc(&c->maps[i].tmap[k], c->prec == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                             3, I.pop[k], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                char msg[64];
                std::snprintf(msg, sizeof msg, "%d", static_cast<int>(r));
                return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed with CUresult %s", msg);
            }
        }
    }
    return LBM_OK;
}

int upload_insts(lbm_ctx* c) {
    CK(c, cudaMemcpyAsync(c->d_inst, c->h.data(), c->n * sizeof(Inst), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// A context of one lattice passes its descriptor by value (kernel argument
// block); refreshed whenever the tensor maps or the parameters change.
template <typename T> void fill_one(lbm_ctx* c, lbm::StepArgs<T>& a, const lbm::Phys<T>& P) {
    const Inst& I = c->h[0];
    a.tmap[0] = c->maps[0].tmap[0];
    a.tmap[1] = c->maps[0].tmap[1];
    a.P = P;
    a.pop[0] = I.pop[0];
    a.pop[1] = I.pop[1];
    a.status = I.status;
    a.plane = I.plane;
    a.nx = I.nx;
    a.ny = I.ny;
    a.pitch = I.pitch;
    a.tiles_x = (I.nx + lbm::step_config(c->prec, c->cfg).bx - 1) / lbm::step_config(c->prec, c->cfg).bx;
}

// The per-instance part of a batched argument block: array addresses and
// sizes, and in FP32 the constants (FP64 kernels read those from the
// descriptors).
template <typename T> void fill_slots(const lbm_ctx* c, lbm::BatchArgs<T>& a) {
    for (int k = 0; k < a.n; ++k) {
        const Inst& I = c->h[a.inst[k]];
        a.lat[k].pop[0] = I.pop[0];
        a.lat[k].pop[1] = I.pop[1];
        a.lat[k].status = I.status;
        a.lat[k].plane = I.plane;
        a.lat[k].nx = I.nx;
        a.lat[k].ny = I.ny;
        a.lat[k].pitch = I.pitch;
        if constexpr (std::is_same<T, float>::value) a.phys.P[k] = I.pf;
    }
}

// Argument blocks after a change of an instance's parameters.
void refresh_args(lbm_ctx* c) {
    for (auto& a : c->rargs_f)
        for (int k = 0; k < a.n; ++k) a.phys.P[k] = c->h[a.inst[k]].pf;
    if (c->n != 1) {
        for (auto& v : c->bargs_f)
            for (auto& a : v) fill_slots(c, a);
        return;
    }
    fill_one(c, c->one_f, c->h[0].pf);
    fill_one(c, c->one_d, c->h[0].pd);
}

const void* one_args(lbm_ctx* c) {
    if (c->n != 1) return nullptr;
    return c->prec == LBM_FP32 ? static_cast<const void*>(&c->one_f) : static_cast<const void*>(&c->one_d);
}

// Tiles and argument blocks for the current tile configuration and schedule.
// Instances are ordered (schedule 0: by index, 1: by index with the tiles of
// each chunk's instances interleaved through a tile table, 2: most tiles
// first) and cut into chunks of kBatchLaunchMax; a chunk's tiles run in slot
// order, row-major within an instance, unless it has a tile table.
template <typename T>
int build_chunks(lbm_ctx* c, std::vector<lbm::BatchArgs<T>> (&out)[2], const std::vector<int>& order,
                 const std::vector<int>& tx, const std::vector<int>& cnt, const lbm::TileCfg& t,
                 std::vector<int4>& table) {
    for (int c0 = 0; c0 < c->n; c0 += lbm::kBatchLaunchMax) {
        const int m = std::min(lbm::kBatchLaunchMax, c->n - c0);
        lbm::BatchArgs<T> a;
        std::memset(&a, 0, sizeof a);
        a.n = m;
        int first = 0;
        for (int k = 0; k < m; ++k) {
            const int i = order[c0 + k];
            a.inst[k] = i;
            a.tiles_x[k] = tx[i];
            lbm::tile_row_magic(tx[i], &a.div_m[k], &a.div_s[k]);
            for (int r = 0; r < cnt[i]; ++r)   // the kernel's row of every tile of the instance
                if (lbm::tile_row(r, a.div_m[k], a.div_s[k]) != r / tx[i])
                    return fail(c, LBM_EINVAL, "tile row by multiplication disagrees with division%s");
            a.first[k] = first;
            first += cnt[i];
        }
        a.first[m] = first;
        fill_slots(c, a);
        if (c->sched == 1) {
            a.tiles = c->d_tiles + table.size();
            int most = 0;
            for (int k = 0; k < m; ++k) most = std::max(most, cnt[a.inst[k]]);
            for (int r = 0; r < most; ++r)
                for (int k = 0; k < m; ++k)
                    if (r < cnt[a.inst[k]])
                        table.push_back(make_int4(k, (r % a.tiles_x[k]) * t.bx, (r / a.tiles_x[k]) * t.by, 0));
        }
        for (int par = 0; par < 2; ++par) {
            for (int k = 0; k < m; ++k) a.tmap[k] = c->maps[a.inst[k]].tmap[par];
            out[par].push_back(a);
        }
        c->chunk_tiles.push_back(first);
    }
    return LBM_OK;
}

// The chunks of the multi-step launches over instances of bytes[i] bytes of
// populations (both time levels): instances largest first (index order
// among equal sizes, so that a chunk holds lattices of one size and its
// tiles per step stay even), cut into as few chunks as kRunMax instances per
// chunk and kRunChunkBytes per chunk allow (an instance larger than that is
// a chunk of its own), with the bytes spread evenly over the chunks.  A
// chunk steps its instances through all the steps of one lbm_step call in
// one launch (instances are independent), so a chunk that fits in L2 (129 MB
// on GB300) keeps its populations there from step to step.  Even chunks
// matter: a last chunk of a few instances has too few tiles per step for
// the resident CTAs, which then wait on its step-to-step dependencies (60
// droplets of 256^2 in chunks of 13 and a last one of 8: 69.7 G updates/s;
// in four chunks of 15: 75.7).  Host arithmetic only.
constexpr size_t kRunChunkBytes = static_cast<size_t>(LBM_RUN_CHUNK_MB) << 20;
std::vector<std::vector<int>> plan_run_chunks(const std::vector<size_t>& bytes) {
    const int n = static_cast<int>(bytes.size());
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return bytes[x] > bytes[y]; });
    auto bytes_of = [&](int j) { return bytes[order[j]]; };
    // the chunk count: as many as filling each chunk up to the limits needs
    size_t left = 0;
    int chunks = 0;
    for (int c0 = 0, m = 0; c0 < n; c0 += m, ++chunks) {
        size_t sum = 0;
        for (m = 0; c0 + m < n && m < lbm::kRunMax; ++m) {
            const size_t b = bytes_of(c0 + m);
            if (m > 0 && sum + b > kRunChunkBytes) break;
            sum += b;
        }
        left += sum;
    }
    std::vector<std::vector<int>> plan;
    for (int c0 = 0, m = 0; c0 < n; c0 += m, --chunks) {
        // this chunk's share of what is left, cut at the instance nearest to it
        const size_t target = left / static_cast<size_t>(std::max(chunks, 1));
        size_t sum = 0;
        for (m = 0; c0 + m < n && m < lbm::kRunMax; ++m) {
            const size_t b = bytes_of(c0 + m);
            if (m > 0 && (sum + b > kRunChunkBytes || sum + b / 2 > target)) break;
            sum += b;
        }
        left -= sum;
        plan.emplace_back(order.begin() + c0, order.begin() + c0 + m);
    }
    return plan;
}

// Argument blocks of the multi-step launches, one per chunk of
// plan_run_chunks.
template <typename T>
int build_run_chunks(lbm_ctx* c, std::vector<lbm::RunArgs<T>>& out, const std::vector<int>& tx,
                     const std::vector<int>& cnt) {
    int* done = reinterpret_cast<int*>(c->d_run + 16);
    std::vector<size_t> bytes(c->n);
    for (int i = 0; i < c->n; ++i) bytes[i] = 2 * 9 * static_cast<size_t>(c->h[i].plane) * c->esz;
    int tile0 = 0;
    for (const std::vector<int>& chunk : plan_run_chunks(bytes)) {
        const int m = static_cast<int>(chunk.size());
        lbm::RunArgs<T> a;
        std::memset(&a, 0, sizeof a);
        a.n = m;
        int first = 0;
        for (int k = 0; k < m; ++k) {
            const int i = chunk[k];
            const Inst& I = c->h[i];
            a.inst[k] = i;
            a.tiles_x[k] = tx[i];
            a.first[k] = first;
            first += cnt[i];
            a.tmap[0][k] = c->maps[i].tmap[0];
            a.tmap[1][k] = c->maps[i].tmap[1];
            a.lat[k].pop[0] = I.pop[0];
            a.lat[k].pop[1] = I.pop[1];
            a.lat[k].status = I.status;
            a.lat[k].plane = I.plane;
            a.lat[k].nx = I.nx;
            a.lat[k].ny = I.ny;
            a.lat[k].pitch = I.pitch;
            if constexpr (std::is_same<T, float>::value) a.phys.P[k] = I.pf;
        }
        a.first[m] = first;
        a.ntiles = first;
        a.done = done + tile0;
        a.counter = reinterpret_cast<unsigned long long*>(c->d_run);
        a.abort_flag = reinterpret_cast<int*>(c->d_run + 8);
        c->run_first.push_back(tile0);
        tile0 += first;
        out.push_back(a);
    }
    return LBM_OK;
}

int build_tiles(lbm_ctx* c) {
    const lbm::TileCfg t = lbm::step_config(c->prec, c->cfg);
    std::vector<int> tx(c->n), cnt(c->n);
    size_t total = 0;
    for (int i = 0; i < c->n; ++i) {
        tx[i] = (c->nx[i] + t.bx - 1) / t.bx;
        cnt[i] = tx[i] * ((c->ny[i] + t.by - 1) / t.by);
        total += static_cast<size_t>(cnt[i]);
    }
    if (total > c->L.tiles_cap || total > 0x7fffffff) return fail(c, LBM_ENOMEM, "tile table larger than reserved%s");
    c->ntiles = static_cast<int>(total);
    for (auto& v : c->bargs_f) v.clear();
    for (auto& v : c->bargs_d) v.clear();
    c->chunk_tiles.clear();
    c->rargs_f.clear();
    c->rargs_d.clear();
    c->run_first.clear();
    if (c->sched == 3)
        return c->prec == LBM_FP32 ? build_run_chunks(c, c->rargs_f, tx, cnt) : build_run_chunks(c, c->rargs_d, tx, cnt);
    if (c->n == 1) return LBM_OK;   // one lattice: StepArgs, tiles from blockIdx

    std::vector<int> order(c->n);
    for (int i = 0; i < c->n; ++i) order[i] = i;
    if (c->sched == 2) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
    std::vector<int4> table;   // schedule 1: every chunk's table, one after another
    const int rc = c->prec == LBM_FP32 ? build_chunks(c, c->bargs_f, order, tx, cnt, t, table)
                                       : build_chunks(c, c->bargs_d, order, tx, cnt, t, table);
    if (rc) return rc;
    if (!table.empty()) {
        CK(c, cudaMemcpyAsync(c->d_tiles, table.data(), table.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

// Kernel launches of one step, and their issue on a stream.
int step_launches(const lbm_ctx* c) { return c->n == 1 ? 1 : static_cast<int>(c->chunk_tiles.size()); }

// n steps of every instance as one multi-step launch per chunk (schedule 3).
template <typename T> int run_steps_t(lbm_ctx* c, std::vector<lbm::RunArgs<T>>& chunks, int n) {
    for (auto& a : chunks) {
        a.nsteps = n;
        a.parity0 = c->parity;
        CK(c, cudaMemsetAsync(c->d_run, 0, 16, c->stream));
        CK(c, cudaMemsetAsync(a.done, 0, static_cast<size_t>(a.ntiles) * sizeof(int), c->stream));
        CK(c, lbm::run_launch(c->prec, c->cfg, c->d_inst, &a, c->n == 1, a.ntiles, n, kTimeoutNs, c->stream));
    }
    return LBM_OK;
}

int run_steps(lbm_ctx* c, int n) {
    if (n <= 0) return LBM_OK;
    const int rc = c->prec == LBM_FP32 ? run_steps_t(c, c->rargs_f, n) : run_steps_t(c, c->rargs_d, n);
    if (rc) return rc;
    c->parity ^= (n & 1);
    c->steps += n;
    c->launches += static_cast<long long>(c->prec == LBM_FP32 ? c->rargs_f.size() : c->rargs_d.size());
    return LBM_OK;
}

cudaError_t launch_step(lbm_ctx* c, int parity) {
    if (c->n == 1)
        return lbm::step_launch(c->prec, c->cfg, c->d_inst, one_args(c), true, c->ntiles, parity, kTimeoutNs,
                                c->stream);
    for (size_t j = 0; j < c->chunk_tiles.size(); ++j) {
        const void* a = c->prec == LBM_FP32 ? static_cast<const void*>(&c->bargs_f[parity][j])
                                            : static_cast<const void*>(&c->bargs_d[parity][j]);
        cudaError_t e = lbm::step_launch(c->prec, c->cfg, c->d_inst, a, false, c->chunk_tiles[j], parity, kTimeoutNs,
                                         c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int apply_schedule(lbm_ctx* c, int cfg, int sched) {
    if (sched == 3 && !lbm::run_supported(c->prec, cfg))
        return fail(c, LBM_EINVAL, "the multi-step schedule needs a tile configuration of one box per CTA%s");
    if (sched == 4 && (c->n != 1 || !lbm::cluster_supported(c->prec, c->nx[0], c->ny[0])))
        return fail(c, LBM_EINVAL, "the cluster schedule needs one lattice that fits one cluster's shared memory%s");
    c->cfg = cfg;
    c->sched = sched;
    drop_graphs(c);
    CK(c, lbm::step_prepare(c->prec, cfg));
    int rc = encode_maps(c);
    if (rc) return rc;
    refresh_args(c);
    rc = upload_insts(c);
    if (rc) return rc;
    return build_tiles(c);
}

template <typename T> void fill_phys(lbm::Phys<T>& P, const HostParams& hp) {
    lbm::fill_eos(P, hp.eos);
    P.flags = hp.flags;
    P.A = T(hp.A);
    P.kappa = T(hp.kappa);
    P.G = T(hp.G);
    P.two_over_G = hp.G != 0.0 ? T(2.0 / hp.G) : T(0);
    P.interact = hp.G != 0.0;
    for (int k = 0; k < 9; ++k) {
        P.s[k] = T(hp.s[k]);
        P.hs[k] = T(1.0 - 0.5 * hp.s[k]);
        P.ns[k] = -P.s[k];
        P.nhs[k] = -P.hs[k];
    }
    P.h2s7 = T(2) * P.hs[7];
    P.h6s1 = T(6.0 * (1.0 - 0.5 * hp.s[1]));
    P.nh6s2 = T(-6.0 * (1.0 - 0.5 * hp.s[2]));
    P.c1 = T(1.5 * hp.s[1]);
    P.c2 = (hp.flags & LBM_FLAG_LI_EPS) ? T(-1.5 * hp.s[2]) : T(0);
    P.rho_ref = T(hp.rho_ref);
    P.var_visc = hp.var_visc;
    P.nu_g = T(hp.nu_g);
    P.dnu = T(hp.nu_l - hp.nu_g);
    P.visc_rho_g = T(hp.visc_rho_g);
    P.visc_inv_drho = hp.var_visc ? T(1.0 / (hp.visc_rho_l - hp.visc_rho_g)) : T(0);
}

int check_idx(lbm_ctx* c, int i) {
    if (!c) return LBM_EINVAL;
    if (i < 0 || i >= c->n) return fail(c, LBM_EINVAL, "instance index out of range%s");
    return LBM_OK;
}

int status_of(lbm_ctx* c, int i, int* code) {
    int st = 0;
    CK(c, cudaMemcpy(&st, c->d_status + i, sizeof(int), cudaMemcpyDeviceToHost));
    *code = (st & lbm::ST_UNSTABLE) ? LBM_EUNSTABLE : ((st & lbm::ST_TIMEOUT) ? LBM_ETIMEOUT : LBM_OK);
    return LBM_OK;
}

int sync_all(lbm_ctx* c) {
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaStreamSynchronize(c->stream));
    std::vector<int> st(c->n);
    CK(c, cudaMemcpy(st.data(), c->d_status, c->n * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < c->n; ++i) {
        if (st[i] & lbm::ST_UNSTABLE) {
            char m[32];
            std::snprintf(m, sizeof m, "%d", i);
            return fail(c, LBM_EUNSTABLE, "instance %s: a density left the psi domain of the EOS or became NaN", m);
        }
        if (st[i] & lbm::ST_TIMEOUT) {
            char m[32];
            std::snprintf(m, sizeof m, "%d", i);
            return fail(c, LBM_ETIMEOUT, "instance %s: a bounded device wait gave up", m);
        }
    }
    return LBM_OK;
}

// n steps of a lattice held in one cluster's shared memory (schedule 4):
// one launch, then the ghost cells of the time level it wrote last.
int cluster_steps(lbm_ctx* c, int n) {
    if (n <= 0) return LBM_OK;
    CK(c, lbm::cluster_run(c->h[0], c->parity, n, c->stream));
    CK(c, lbm::aux_fill_ghosts(c->h[0], c->d_inst, c->parity ^ (n & 1), c->stream));
    c->parity ^= (n & 1);
    c->steps += n;
    c->launches += 1;
    return LBM_OK;
}

int launch_steps(lbm_ctx* c, int n) {
    if (c->sched == 3) return run_steps(c, n);
    if (c->sched == 4) return cluster_steps(c, n);
    for (int k = 0; k < n; ++k) {
        CK(c, launch_step(c, c->parity));
        c->parity ^= 1;
        c->launches += step_launches(c);
        ++c->steps;
    }
    return LBM_OK;
}

// The graph of 2 << level steps from time level `parity`, captured (not
// run) on first use.
int ensure_graph(lbm_ctx* c, int parity, int level) {
    if (c->gexec[parity][level]) return LBM_OK;
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < (2 << level); ++k) {
        cudaError_t e = launch_step(c, parity ^ (k & 1));
        if (e != cudaSuccess) {
            g = nullptr;
            if (cudaStreamEndCapture(c->stream, &g) == cudaSuccess && g) cudaGraphDestroy(g);
            return cuda_fail(c, e, "step launch during graph capture");
        }
    }
    CK(c, cudaStreamEndCapture(c->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&c->gexec[parity][level], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    return LBM_OK;
}

int ready(lbm_ctx* c) {
    for (int i = 0; i < c->n; ++i) {
        if (!c->hp[i].set) return fail(c, LBM_EINVAL, "parameters of an instance were never set%s");
        if (!c->inited[i]) return fail(c, LBM_EINVAL, "an instance was never initialised%s");
    }
    return LBM_OK;
}

int valid_params(const lbm_eos* eos, double A, double kappa, double G, const double* s, double rho_ref) {
    if (!lbm::eos_valid_at(eos) || !s) return 0;
    if (!std::isfinite(A) || !std::isfinite(kappa) || !std::isfinite(G) || !std::isfinite(rho_ref)) return 0;
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(s[k]) || s[k] <= 0.0 || s[k] >= 2.0) return 0;
    return 1;
}

}  // namespace

// =========================================================================
namespace {
// Initial state from host fields of R (double, or float widened exactly).
// Row bands of a field moved between host and device: a lattice of 2^20
// nodes or more in kReadBands bands (each band's copy overlapping another
// band's kernel), a smaller one whole.
int field_bands(const lbm_ctx* c, int i) {
    const size_t N = static_cast<size_t>(c->nx[i]) * c->ny[i];
    return N >= kReadBandMin && c->ny[i] >= kReadBands ? kReadBands : 1;
}

// The second stream of the banded copies and its per-band events, created
// once, whole or not at all.
int ensure_copy_stream(lbm_ctx* c) {
    if (c->copy_stream) return LBM_OK;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kReadBands] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int b = 0; b < kReadBands && e == cudaSuccess; ++b)
        e = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        if (cs) cudaStreamDestroy(cs);
        return cuda_fail(c, e, "copy stream of the banded field transfers");
    }
    c->copy_stream = cs;
    std::copy(ev, ev + kReadBands, c->band_done);
    return LBM_OK;
}

template <typename R> int init_density_t(lbm_ctx* c, int i, const R* rho, const R* ux, const R* uy) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!rho) return fail(c, LBM_EINVAL, "rho must not be NULL%s");
    if (!c->hp[i].set) return fail(c, LBM_EINVAL, "set the parameters before the density%s");
    Range range("lbm_batch_init_density");
    const size_t N = static_cast<size_t>(c->nx[i]) * c->ny[i];
    // the EOS range only matters when psi is evaluated (G != 0)
    const double rmax = c->hp[i].G != 0.0 ? eos_rho_max(c->hp[i].eos) : HUGE_VAL;
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaStreamSynchronize(c->stream));
    R* const scratch = reinterpret_cast<R*>(c->d_scratch);
    R* d_rho = scratch;
    R* d_ux = ux ? scratch + N : nullptr;
    R* d_uy = uy ? scratch + 2 * N : nullptr;
    constexpr bool f32 = sizeof(R) == 4;
    // the field is checked on the device before anything of the instance's
    // current time level is written.  One lattice of 2^20 nodes or more: the
    // field arrives in row bands on the copy stream, each band checked and
    // its equilibrium written into the other time level (which the next step
    // overwrites whole) while the next band is in flight; that level becomes
    // the current one once the whole field has passed.
    int* d_bad = reinterpret_cast<int*>(c->d_result);
    int bad = 0;
    const int bands = c->n == 1 ? field_bands(c, i) : 1;
    const int level = bands > 1 ? c->parity ^ 1 : c->parity;
    if (bands > 1 && (rc = ensure_copy_stream(c))) return rc;
    auto copy_and_check = [&]() -> int {
        CK(c, cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
        if (bands == 1) {
            CK(c, cudaMemcpyAsync(d_rho, rho, N * sizeof(R), cudaMemcpyHostToDevice, c->stream));
            if (ux) CK(c, cudaMemcpyAsync(d_ux, ux, N * sizeof(R), cudaMemcpyHostToDevice, c->stream));
            if (uy) CK(c, cudaMemcpyAsync(d_uy, uy, N * sizeof(R), cudaMemcpyHostToDevice, c->stream));
            CK(c, lbm::aux_check_init(d_rho, d_ux, d_uy, f32, static_cast<long long>(N), rmax, d_bad, c->stream));
        } else {
            const int nx = c->nx[i], ny = c->ny[i];
            for (int b = 0; b < bands; ++b) {
                const int y0 = static_cast<int>(static_cast<long long>(ny) * b / bands);
                const int y1 = static_cast<int>(static_cast<long long>(ny) * (b + 1) / bands);
                const size_t off = static_cast<size_t>(y0) * nx, cnt = static_cast<size_t>(y1 - y0) * nx;
                CK(c, cudaMemcpyAsync(d_rho + off, rho + off, cnt * sizeof(R), cudaMemcpyHostToDevice, c->copy_stream));
                if (ux)
                    CK(c, cudaMemcpyAsync(d_ux + off, ux + off, cnt * sizeof(R), cudaMemcpyHostToDevice,
                                          c->copy_stream));
                if (uy)
                    CK(c, cudaMemcpyAsync(d_uy + off, uy + off, cnt * sizeof(R), cudaMemcpyHostToDevice,
                                          c->copy_stream));
                CK(c, cudaEventRecord(c->band_done[b], c->copy_stream));
                CK(c, cudaStreamWaitEvent(c->stream, c->band_done[b], 0));
                CK(c, lbm::aux_check_init(d_rho + off, d_ux ? d_ux + off : nullptr, d_uy ? d_uy + off : nullptr, f32,
                                          static_cast<long long>(cnt), rmax, d_bad, c->stream));
                CK(c, lbm::aux_init_rows(c->h[i], c->d_inst + i, d_rho, d_ux, d_uy, f32, level, y0, y1, c->stream));
            }
        }
        CK(c, cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        return LBM_OK;
    };
    rc = copy_and_check();
    if (rc) {   // no copy from the caller's arrays (or into `bad`) may outlive the call
        if (bands > 1) cudaStreamSynchronize(c->copy_stream);
        cudaStreamSynchronize(c->stream);
        return rc;
    }
    // the stream waited for every band's copy: all of them have landed
    CK(c, cudaStreamSynchronize(c->stream));
    if (bad & 1) return fail(c, LBM_EINVAL, "initial density must be finite, positive and inside the EOS range%s");
    if (bad & 2) return fail(c, LBM_EINVAL, "initial velocity must be finite%s");
    if (bands == 1) {
        CK(c, lbm::aux_init(c->h[i], c->d_inst + i, d_rho, d_ux, d_uy, f32, c->parity, c->stream));
    } else {
        CK(c, lbm::aux_fill_ghosts(c->h[i], c->d_inst + i, level, c->stream));
        c->parity = level;
    }
    CK(c, cudaMemsetAsync(c->d_status + i, 0, sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->inited[i] = 1;
    c->steps = 0;
    return LBM_OK;
}

// Macroscopic fields into host arrays of O (double, or float: each value
// rounded to nearest).
template <typename O> int read_fields_t(lbm_ctx* c, int i, O* rho, O* ux, O* uy, O* psi) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!c->inited[i] || !c->hp[i].set) return fail(c, LBM_EINVAL, "instance not initialised%s");
    Range range("lbm_batch_read_fields");
    CK(c, cudaSetDevice(c->device));
    const int nx = c->nx[i], ny = c->ny[i];
    const size_t N = static_cast<size_t>(nx) * ny;
    // a large lattice in row bands: band b's copy to the host overlaps band b + 1's kernel
    const int bands = field_bands(c, i);
    if (bands > 1 && (rc = ensure_copy_stream(c))) return rc;
    O* outs[4] = {rho, ux, uy, psi};
    O* const scratch = reinterpret_cast<O*>(c->d_scratch);
    constexpr bool f32 = sizeof(O) == 4;
    for (int f = 0; f < 4; ++f) {
        if (!outs[f]) continue;
        if (bands == 1) {
            CK(c, lbm::aux_field(c->h[i], c->d_inst + i, c->parity, f, 0, ny, scratch, f32, c->stream));
            CK(c, cudaMemcpyAsync(outs[f], scratch, N * sizeof(O), cudaMemcpyDeviceToHost, c->stream));
            CK(c, cudaStreamSynchronize(c->stream));
            continue;
        }
        auto issue_bands = [&]() -> int {
            for (int b = 0; b < bands; ++b) {
                const int y0 = static_cast<int>(static_cast<long long>(ny) * b / bands);
                const int y1 = static_cast<int>(static_cast<long long>(ny) * (b + 1) / bands);
                const size_t off = static_cast<size_t>(y0) * nx, cnt = static_cast<size_t>(y1 - y0) * nx;
                CK(c, lbm::aux_field(c->h[i], c->d_inst + i, c->parity, f, y0, y1, scratch, f32, c->stream));
                CK(c, cudaEventRecord(c->band_done[b], c->stream));
                CK(c, cudaStreamWaitEvent(c->copy_stream, c->band_done[b], 0));
                CK(c, cudaMemcpyAsync(outs[f] + off, scratch + off, cnt * sizeof(O), cudaMemcpyDeviceToHost,
                                      c->copy_stream));
            }
            return LBM_OK;
        };
        rc = issue_bands();
        if (rc) {   // no copy into the caller's array may outlive the call
            cudaStreamSynchronize(c->copy_stream);
            return rc;
        }
        CK(c, cudaStreamSynchronize(c->copy_stream));   // before the next field reuses the scratch
    }
    int code = LBM_OK;
    rc = status_of(c, i, &code);
    return rc ? rc : code;
}

}  // namespace

extern "C" {

int lbm_eos_pressure(const lbm_eos* eos, double rho, double* p) {
    if (!eos_valid(eos) || !p || !(rho >= 0)) return LBM_EINVAL;
    *p = eos_p(*eos, rho);
    return LBM_OK;
}

int lbm_eos_critical(const lbm_eos* eos, double* rho_c, double* T_c, double* p_c) {
    if (!eos_valid(eos)) return LBM_EINVAL;
    lbm_eos e = *eos;
    const double hi = eos_rho_max(e);
    auto min_slope = [&](double T, double* arg) {
        e.T = T;
        double fm;
        *arg = golden_min([&](double r) { return eos_dp(e, r); }, 1e-9 * hi, 0.999 * hi, &fm);
        return fm;
    };
    double lo = 1e-9, up = 1.0, arg;
    for (int it = 0; it < 200 && min_slope(up, &arg) <= 0; ++it) up *= 2.0;
    const double Tc = bisect([&](double T) { double a2; return min_slope(T, &a2); }, lo, up);
    min_slope(Tc, &arg);
    e.T = Tc;
    if (rho_c) *rho_c = arg;
    if (T_c) *T_c = Tc;
    if (p_c) *p_c = eos_p(e, arg);
    return LBM_OK;
}

int lbm_eos_maxwell(const lbm_eos* eos, double* rho_g, double* rho_l, double* p0_out) {
    if (!lbm::eos_valid_at(eos)) return LBM_EINVAL;
    const lbm_eos& e = *eos;
    const double hi = eos_rho_max(e);
    double fm;
    const double rm = golden_min([&](double r) { return eos_dp(e, r); }, 1e-9 * hi, 0.999 * hi, &fm);
    if (!(fm < 0)) return LBM_EINVAL;   // not below the critical temperature
    const double s1 = bisect([&](double r) { return eos_dp(e, r); }, 1e-12 * hi, rm);
    const double s2 = bisect([&](double r) { return -eos_dp(e, r); }, rm, 0.99999 * hi);
    const double p_hi = eos_p(e, s1), p_lo = std::max(eos_p(e, s2), 0.0);
    auto roots = [&](double p0, double* rg, double* rl) {
        *rg = bisect([&](double r) { return eos_p(e, r) - p0; }, 0.0, s1);
        *rl = bisect([&](double r) { return eos_p(e, r) - p0; }, s2, 0.99999999 * hi);
    };
    auto area = [&](double p0) {
        double rg, rl;
        roots(p0, &rg, &rl);
        return gauss_int(e, p0, rg, s1, 256) + gauss_int(e, p0, s1, s2, 256) + gauss_int(e, p0, s2, rl, 256);
    };
    const double span = p_hi - p_lo;
    double a = p_lo + 1e-12 * span, b = p_hi - 1e-12 * span;
    double fa = area(a);
    if (!((fa < 0) != (area(b) < 0))) return LBM_EINVAL;
    for (int it = 0; it < 200; ++it) {
        const double m = 0.5 * (a + b);
        if (m <= a || m >= b) break;
        const double fmid = area(m);
        if ((fmid < 0) == (fa < 0)) { a = m; fa = fmid; } else { b = m; }
    }
    const double p0 = 0.5 * (a + b);
    double rg, rl;
    roots(p0, &rg, &rl);
    if (rho_g) *rho_g = rg;
    if (rho_l) *rho_l = rl;
    if (p0_out) *p0_out = p0;
    return LBM_OK;
}

int lbm_fp64_math_check(double lo, double hi, long long n, unsigned long long result[4]) {
    if (!result || n < 1 || !(lo > 0.0) || !(hi > lo) || !std::isfinite(hi)) return LBM_EINVAL;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    int rc = LBM_OK;
    if (cudaMemset(d, 0, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        lbm::aux_math_check(n, lo, hi, d) != cudaSuccess ||
        cudaMemcpy(result, d, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        rc = LBM_ECUDA;
    }
    cudaFree(d);
    return rc;
}

int lbm_fp64_fma_rate(int iters, void* stream, double* flops_per_s, double* seconds) {
    if (iters < 1 || !flops_per_s || !seconds) return LBM_EINVAL;
    if (lbm::aux_fp64_fma_rate(iters, static_cast<cudaStream_t>(stream), flops_per_s, seconds) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    return LBM_OK;
}

int lbm_laplace_fit(int n, const double* dp, const double* R, double* sigma, double* icpt, double* r2) {
    if (n < 2 || !dp || !R) return LBM_EINVAL;
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int i = 0; i < n; ++i) {
        if (!(R[i] > 0)) return LBM_EINVAL;
        const double x = 1.0 / R[i];
        sx += x; sy += dp[i]; sxx += x * x; sxy += x * dp[i];
    }
    const double den = n * sxx - sx * sx;
    if (den == 0.0) return LBM_EINVAL;
    const double k = (n * sxy - sx * sy) / den, c = (sy - k * sx) / n;
    double ssr = 0, sst = 0;
    const double ym = sy / n;
    for (int i = 0; i < n; ++i) {
        const double y = k / R[i] + c;
        ssr += (dp[i] - y) * (dp[i] - y);
        sst += (dp[i] - ym) * (dp[i] - ym);
    }
    if (sigma) *sigma = k;
    if (icpt) *icpt = c;
    if (r2) *r2 = sst > 0 ? 1.0 - ssr / sst : 1.0;
    return LBM_OK;
}

size_t lbm_batch_required_bytes(int n, const int* nx, const int* ny, int precision) {
    if (!valid_shape(n, nx, ny, precision)) return 0;
    return make_layout(n, nx, ny, precision).total;
}

size_t lbm_required_bytes(int nx, int ny, int precision) { return lbm_batch_required_bytes(1, &nx, &ny, precision); }

int lbm_run_chunk_plan(int n, const int* nx, const int* ny, int precision, int* chunk_of) {
    if (!valid_shape(n, nx, ny, precision) || !chunk_of) return LBM_EINVAL;
    std::vector<size_t> bytes(n);
    for (int i = 0; i < n; ++i)
        bytes[i] = 2 * 9 * static_cast<size_t>(pitch_of(nx[i], precision)) * (ny[i] + 2 * lbm::GY) * esize(precision);
    const std::vector<std::vector<int>> plan = plan_run_chunks(bytes);
    for (size_t k = 0; k < plan.size(); ++k)
        for (int i : plan[k]) chunk_of[i] = static_cast<int>(k);
    return static_cast<int>(plan.size());
}

int lbm_batch_create(lbm_ctx** out, int n, const int* nx, const int* ny, int precision, void* dev_buf,
                     size_t buf_bytes, void* stream) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!valid_shape(n, nx, ny, precision)) return LBM_EINVAL;
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) % 256) != 0) return LBM_EINVAL;
    lbm_ctx* c = new lbm_ctx();
    c->n = n;
    c->prec = precision;
    c->esz = esize(precision);
    c->nx.assign(nx, nx + n);
    c->ny.assign(ny, ny + n);
    c->L = make_layout(n, nx, ny, precision);
    c->stream = static_cast<cudaStream_t>(stream);
    c->hp.assign(n, HostParams{});
    c->inited.assign(n, 0);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return LBM_ECUDA;
    }
    if (dev_buf) {
        if (buf_bytes < c->L.total) {
            delete c;
            return LBM_ENOMEM;
        }
        c->buf = static_cast<char*>(dev_buf);
        c->buf_bytes = buf_bytes;
    } else {
        if (cudaMalloc(&c->buf, c->L.total) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return LBM_ENOMEM;
        }
        c->owns = true;
        c->buf_bytes = c->L.total;
    }
    if (cudaMemsetAsync(c->buf, 0, c->L.total, c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        lbm_destroy(c);
        return LBM_ECUDA;
    }
    c->d_inst = reinterpret_cast<Inst*>(c->buf + c->L.inst_off);
    c->d_tiles = reinterpret_cast<int4*>(c->buf + c->L.tiles_off);
    c->d_status = reinterpret_cast<int*>(c->buf + c->L.status_off);
    c->d_partials = reinterpret_cast<double*>(c->buf + c->L.partials_off);
    c->d_result = reinterpret_cast<double*>(c->buf + c->L.result_off);
    c->d_scratch = reinterpret_cast<double*>(c->buf + c->L.scratch_off);
    c->d_run = c->buf + c->L.run_off;
    c->h.assign(n, Inst{});
    c->maps.assign(n, Maps{});
    for (int i = 0; i < n; ++i) {
        Inst& I = c->h[i];
        std::memset(&I, 0, sizeof(Inst));
        I.pop[0] = c->buf + c->L.pop_off[0][i];
        I.pop[1] = c->buf + c->L.pop_off[1][i];
        I.status = c->d_status + i;
        I.nx = nx[i];
        I.ny = ny[i];
        I.pitch = pitch_of(nx[i], precision);
        I.nyp = ny[i] + 2 * lbm::GY;
        I.plane = static_cast<long long>(I.pitch) * I.nyp;
        I.prec = precision;
    }
    int rc = apply_schedule(c, 0, 0);
    if (rc) {
        lbm_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

int lbm_create(lbm_ctx** out, int nx, int ny, int precision, void* dev_buf, size_t buf_bytes, void* stream) {
    return lbm_batch_create(out, 1, &nx, &ny, precision, dev_buf, buf_bytes, stream);
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream || c->buf) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    for (auto& e : c->band_done)
        if (e) cudaEventDestroy(e);
    if (c->owns && c->buf) cudaFree(c->buf);
    delete c;
}

int lbm_batch_set_params(lbm_ctx* c, int i, const lbm_eos* eos, double A, double kappa, double G, const double s[9],
                         double rho_ref, unsigned flags) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!valid_params(eos, A, kappa, G, s, rho_ref)) return fail(c, LBM_EINVAL, "invalid model parameters%s");
    CK(c, cudaSetDevice(c->device));
    HostParams& hp = c->hp[i];
    const HostParams keep = hp;
    hp.eos = *eos;
    hp.A = A;
    hp.kappa = kappa;
    hp.G = G;
    std::memcpy(hp.s, s, sizeof hp.s);
    hp.rho_ref = rho_ref;
    hp.flags = flags;
    hp.set = 1;
    hp.var_visc = keep.set ? keep.var_visc : 0;   // the viscosity law survives a parameter change
    hp.nu_g = keep.nu_g;
    hp.nu_l = keep.nu_l;
    hp.visc_rho_g = keep.visc_rho_g;
    hp.visc_rho_l = keep.visc_rho_l;
    fill_phys(c->h[i].pf, hp);
    fill_phys(c->h[i].pd, hp);
    refresh_args(c);
    drop_graphs(c);
    return upload_insts(c);
}

int lbm_set_params(lbm_ctx* c, const lbm_eos* eos, double A, double kappa, double G, const double s[9], double rho_ref,
                   unsigned flags) {
    return lbm_batch_set_params(c, 0, eos, A, kappa, G, s, rho_ref, flags);
}

int lbm_batch_set_viscosity(lbm_ctx* c, int i, int enable, double nu_gas, double nu_liquid, double rho_gas,
                            double rho_liquid) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!c->hp[i].set) return fail(c, LBM_EINVAL, "set the parameters before the viscosity law%s");
    if (enable && (!(nu_gas > 0) || !(nu_liquid > 0) || !(rho_liquid > rho_gas) || !std::isfinite(rho_liquid) ||
                   !std::isfinite(nu_gas + nu_liquid + rho_gas)))
        return fail(c, LBM_EINVAL, "viscosities must be positive and rho_liquid > rho_gas%s");
    CK(c, cudaSetDevice(c->device));
    HostParams& hp = c->hp[i];
    hp.var_visc = enable ? 1 : 0;
    hp.nu_g = nu_gas;
    hp.nu_l = nu_liquid;
    hp.visc_rho_g = rho_gas;
    hp.visc_rho_l = rho_liquid;
    fill_phys(c->h[i].pf, hp);
    fill_phys(c->h[i].pd, hp);
    refresh_args(c);
    drop_graphs(c);
    return upload_insts(c);
}

int lbm_set_viscosity(lbm_ctx* c, int enable, double nu_gas, double nu_liquid, double rho_gas, double rho_liquid) {
    return lbm_batch_set_viscosity(c, 0, enable, nu_gas, nu_liquid, rho_gas, rho_liquid);
}


int lbm_batch_init_density(lbm_ctx* c, int i, const double* rho, const double* ux, const double* uy) {
    return init_density_t(c, i, rho, ux, uy);
}
int lbm_batch_init_density_f32(lbm_ctx* c, int i, const float* rho, const float* ux, const float* uy) {
    return init_density_t(c, i, rho, ux, uy);
}
int lbm_init_density(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    return init_density_t(c, 0, rho, ux, uy);
}
int lbm_init_density_f32(lbm_ctx* c, const float* rho, const float* ux, const float* uy) {
    return init_density_t(c, 0, rho, ux, uy);
}

// n steps as lbm_step issues them.  With graphs on (one-step schedules):
// replays of the 32-step graph, then of the 16-, 8-, 4- and 2-step graphs
// the rest's binary digits call for (20 steps: two replays), and a last odd
// step as a plain launch; every graph has an even number of steps, so the
// parity a replay starts from is the current one.
int step_n(lbm_ctx* c, int n) {
    if (c->use_graphs && c->sched < 3) {
        for (int level = kGraphLevels - 1; level >= 0; --level) {
            const int len = 2 << level;
            while (n >= len && (level == kGraphLevels - 1 || n < 2 * len)) {
                int rc = ensure_graph(c, c->parity, level);
                if (rc) return rc;
                Range replay("lbm_step: graph replay");
                CK(c, cudaGraphLaunch(c->gexec[c->parity][level], c->stream));
                c->launches += static_cast<long long>(len) * step_launches(c);
                c->steps += len;
                n -= len;
            }
        }
    }
    return launch_steps(c, n);
}

int lbm_step(lbm_ctx* c, int n) {
    if (!c || n < 0) return LBM_EINVAL;
    Range range("lbm_step");
    int rc = ready(c);
    if (rc) return rc;
    CK(c, cudaSetDevice(c->device));
    return step_n(c, n);
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    return sync_all(c);
}

int lbm_status(lbm_ctx* c, int i) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaStreamSynchronize(c->stream));
    int code = LBM_OK;
    rc = status_of(c, i, &code);
    return rc ? rc : code;
}

int lbm_clear_status(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaMemsetAsync(c->d_status, 0, c->n * sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}


int lbm_batch_read_fields(lbm_ctx* c, int i, double* rho, double* ux, double* uy, double* psi) {
    return read_fields_t(c, i, rho, ux, uy, psi);
}
int lbm_batch_read_fields_f32(lbm_ctx* c, int i, float* rho, float* ux, float* uy, float* psi) {
    return read_fields_t(c, i, rho, ux, uy, psi);
}
int lbm_read_fields(lbm_ctx* c, double* rho, double* ux, double* uy, double* psi) {
    return read_fields_t(c, 0, rho, ux, uy, psi);
}
int lbm_read_fields_f32(lbm_ctx* c, float* rho, float* ux, float* uy, float* psi) {
    return read_fields_t(c, 0, rho, ux, uy, psi);
}

int lbm_batch_read_populations(lbm_ctx* c, int i, double* f) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!f) return fail(c, LBM_EINVAL, "f must not be NULL%s");
    if (!c->inited[i]) return fail(c, LBM_EINVAL, "instance not initialised%s");
    CK(c, cudaSetDevice(c->device));
    const size_t N = static_cast<size_t>(c->nx[i]) * c->ny[i];
    for (int a = 0; a < 9; ++a) {
        CK(c, lbm::aux_gather_plane(c->h[i], c->d_inst + i, c->parity, a, c->d_scratch, c->stream));
        CK(c, cudaMemcpyAsync(f + a * N, c->d_scratch, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    int code = LBM_OK;
    rc = status_of(c, i, &code);
    return rc ? rc : code;
}

int lbm_read_populations(lbm_ctx* c, double* f) { return lbm_batch_read_populations(c, 0, f); }

int lbm_batch_measure(lbm_ctx* c, int i, double cxc, double cyc, double r_in, double r_out, double* out) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!out || !(r_in >= 0) || !(r_out >= 0)) return fail(c, LBM_EINVAL, "bad measurement arguments%s");
    if (!c->inited[i] || !c->hp[i].set) return fail(c, LBM_EINVAL, "instance not initialised%s");
    Range range("lbm_batch_measure");
    CK(c, cudaSetDevice(c->device));
    CK(c, lbm::aux_measure(c->h[i], c->d_inst + i, c->parity, cxc, cyc, r_in, r_out, c->d_partials, c->d_result,
                           c->stream));
    double s[lbm::kReduceSlots];
    CK(c, cudaMemcpyAsync(s, c->d_result, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double N = static_cast<double>(c->nx[i]) * c->ny[i];
    const double p_in = s[3] > 0 ? s[1] / s[3] : NAN, rho_in = s[3] > 0 ? s[2] / s[3] : NAN;
    const double p_out = s[6] > 0 ? s[4] / s[6] : NAN, rho_out = s[6] > 0 ? s[5] / s[6] : NAN;
    const double ex = s[0] - rho_out * N;
    const double R_eq = std::sqrt(std::max(ex, 0.0) / (M_PI * (rho_in - rho_out)));
    const double vals[LBM_MEASURE_N] = {p_in, p_out, rho_in, rho_out, R_eq, s[0], s[3], s[6]};
    std::memcpy(out, vals, sizeof vals);
    int code = LBM_OK;
    rc = status_of(c, i, &code);
    return rc ? rc : code;
}

int lbm_measure_pressure_jump(lbm_ctx* c, double cxc, double cyc, double r_in, double r_out, double* p_in,
                              double* p_out, double* R_eq) {
    double o[LBM_MEASURE_N];
    int rc = lbm_batch_measure(c, 0, cxc, cyc, r_in, r_out, o);
    if (rc == LBM_OK || rc == LBM_EUNSTABLE || rc == LBM_ETIMEOUT) {
        if (p_in) *p_in = o[0];
        if (p_out) *p_out = o[1];
        if (R_eq) *R_eq = o[4];
    }
    return rc;
}

int lbm_batch_stats(lbm_ctx* c, int i, double* out5) {
    int rc = check_idx(c, i);
    if (rc) return rc;
    if (!out5) return fail(c, LBM_EINVAL, "out must not be NULL%s");
    if (!c->inited[i] || !c->hp[i].set) return fail(c, LBM_EINVAL, "instance not initialised%s");
    Range range("lbm_batch_stats");
    CK(c, cudaSetDevice(c->device));
    CK(c, lbm::aux_stats(c->h[i], c->d_inst + i, c->parity, c->d_partials, c->d_result, c->stream));
    double s[lbm::kReduceSlots];
    CK(c, cudaMemcpyAsync(s, c->d_result, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memcpy(out5, s, 5 * sizeof(double));
    int code = LBM_OK;
    rc = status_of(c, i, &code);
    return rc ? rc : code;
}

int lbm_stats(lbm_ctx* c, double* mass, double* mom_x, double* mom_y, double* ke, double* umax) {
    double o[5];
    int rc = lbm_batch_stats(c, 0, o);
    if (rc == LBM_OK || rc == LBM_EUNSTABLE || rc == LBM_ETIMEOUT) {
        if (mass) *mass = o[0];
        if (mom_x) *mom_x = o[1];
        if (mom_y) *mom_y = o[2];
        if (ke) *ke = o[3];
        if (umax) *umax = o[4];
    }
    return rc;
}

// ---- checkpoints ----------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int version, n, prec, pad;
    long long steps;
};
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    int rc = ready(c);
    if (rc) return rc;
    rc = sync_all(c);
    if (rc) return rc;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBM_EIO, "cannot open %s for writing", path);
    CkptHeader hd{};
    std::memcpy(hd.magic, "LBMCKPT1", 8);
    hd.version = 2;
    hd.n = c->n;
    hd.prec = c->prec;
    hd.steps = c->steps;
    bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1;
    for (int i = 0; i < c->n && ok; ++i) {
        int dims[2] = {c->nx[i], c->ny[i]};
        ok = std::fwrite(dims, sizeof dims, 1, fp) == 1 && std::fwrite(&c->hp[i], sizeof(HostParams), 1, fp) == 1;
        const size_t bytes = 9 * static_cast<size_t>(c->h[i].plane) * c->esz;
        std::vector<char> host(bytes);
        if (cudaMemcpy(host.data(), c->h[i].pop[c->parity], bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(fp);
            return fail(c, LBM_ECUDA, "device-to-host copy of the populations failed%s");
        }
        ok = ok && std::fwrite(host.data(), 1, bytes, fp) == bytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(c, LBM_EIO, "writing %s failed", path);
}

int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->device));
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBM_EIO, "cannot open %s", path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, "LBMCKPT1", 8) != 0 || hd.version != 2 ||
        hd.n != c->n || hd.prec != c->prec) {
        std::fclose(fp);
        return fail(c, LBM_EIO, "%s is not a checkpoint of this context's shape and precision", path);
    }
    CK(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->n; ++i) {
        int dims[2];
        HostParams hp;
        if (std::fread(dims, sizeof dims, 1, fp) != 1 || dims[0] != c->nx[i] || dims[1] != c->ny[i] ||
            std::fread(&hp, sizeof hp, 1, fp) != 1) {
            std::fclose(fp);
            return fail(c, LBM_EIO, "%s does not match this context", path);
        }
        const size_t bytes = 9 * static_cast<size_t>(c->h[i].plane) * c->esz;
        std::vector<char> host(bytes);
        if (std::fread(host.data(), 1, bytes, fp) != bytes) {
            std::fclose(fp);
            return fail(c, LBM_EIO, "%s is truncated", path);
        }
        c->hp[i] = hp;
        fill_phys(c->h[i].pf, hp);
        fill_phys(c->h[i].pd, hp);
        if (cudaMemcpy(c->h[i].pop[c->parity], host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(fp);
            return fail(c, LBM_ECUDA, "host-to-device copy of the populations failed%s");
        }
        c->inited[i] = 1;
    }
    std::fclose(fp);
    c->steps = hd.steps;
    refresh_args(c);
    drop_graphs(c);
    CK(c, cudaMemset(c->d_status, 0, c->n * sizeof(int)));
    return upload_insts(c);
}

// ---- tiles, schedules, autotuning ----------------------------------------
int lbm_tile_config_count(int precision) {
    if (esize(precision) == 0) return LBM_EINVAL;
    return lbm::step_config_count(precision);
}

int lbm_tile_config(int precision, int k, int* bx, int* by, int* threads, int* stages) {
    if (esize(precision) == 0 || k < 0 || k >= lbm::step_config_count(precision)) return LBM_EINVAL;
    const lbm::TileCfg t = lbm::step_config(precision, k);
    if (bx) *bx = t.bx;
    if (by) *by = t.by;
    if (threads) *threads = t.threads;
    if (stages) *stages = t.stages;
    return LBM_OK;
}

int lbm_set_schedule(lbm_ctx* c, int tile_config, int schedule) {
    if (!c) return LBM_EINVAL;
    if (tile_config < 0 || tile_config >= lbm::step_config_count(c->prec) || schedule < 0 || schedule >= lbm::kMaxSched)
        return fail(c, LBM_EINVAL, "unknown tile configuration or schedule%s");
    CK(c, cudaSetDevice(c->device));
    CK(c, cudaStreamSynchronize(c->stream));
    return apply_schedule(c, tile_config, schedule);
}

int lbm_autotune(lbm_ctx* c, int steps, int* tile_config, int* schedule, double* ms_per_step) {
    if (!c || steps < 1) return LBM_EINVAL;
    Range range("lbm_autotune");
    int rc = ready(c);
    if (rc) return rc;
    rc = sync_all(c);
    if (rc) return rc;
    // snapshot every instance's current time level, the counters and the status
    std::vector<std::vector<char>> snap(c->n);
    for (int i = 0; i < c->n; ++i) {
        const size_t bytes = 9 * static_cast<size_t>(c->h[i].plane) * c->esz;
        snap[i].resize(bytes);
        CK(c, cudaMemcpy(snap[i].data(), c->h[i].pop[c->parity], bytes, cudaMemcpyDeviceToHost));
    }
    const int parity0 = c->parity;
    const long long steps0 = c->steps, launches0 = c->launches;
    // every candidate is timed the way lbm_step will run it: with graphs on,
    // over whole graph replays (the step count rounded up to kGraphSteps),
    // after a warm-up that captures the graph
    if (c->use_graphs) steps = (steps + kGraphSteps - 1) / kGraphSteps * kGraphSteps;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, LBM_ECUDA, "cudaEventCreate failed%s");
    }
    const int cfg0 = c->cfg, sched0 = c->sched;
    double best = 1e300;
    int bc = cfg0, bs = sched0;
    // one candidate: warm-up (which captures its graphs), then the timed
    // steps; one whose bounded waits gave up (a launch that ended early) is
    // not a candidate
    std::vector<int> st(c->n);
    auto time_one = [&](int k, int s, float* ms, bool* timed_out) -> int {
        int r = apply_schedule(c, k, s);
        if (!r) r = step_n(c, c->use_graphs && s < 3 ? kGraphSteps : 2);
        if (r) return r;
        CK(c, cudaEventRecord(e0, c->stream));
        r = step_n(c, steps);
        if (r) return r;
        CK(c, cudaEventRecord(e1, c->stream));
        CK(c, cudaEventSynchronize(e1));
        CK(c, cudaEventElapsedTime(ms, e0, e1));
        CK(c, cudaMemcpy(st.data(), c->d_status, c->n * sizeof(int), cudaMemcpyDeviceToHost));
        *timed_out = std::any_of(st.begin(), st.end(), [](int v) { return (v & lbm::ST_TIMEOUT) != 0; });
        CK(c, cudaMemset(c->d_status, 0, c->n * sizeof(int)));
        return LBM_OK;
    };
    for (int k = 0; k < lbm::step_config_count(c->prec) && !rc; ++k)
        for (int s = 0; s < lbm::kMaxSched && !rc; ++s) {
            // one lattice: the one-step launch (0), the multi-step one (3) or
            // the cluster (4, one tile configuration stands for all)
            if ((c->n == 1 && s != 0 && s < 3) || (s == 3 && !lbm::run_supported(c->prec, k))) continue;
            if (s == 4 && (k > 0 || c->n != 1 || !lbm::cluster_supported(c->prec, c->nx[0], c->ny[0]))) continue;
            float ms = 0;
            bool timed_out = false;
            rc = time_one(k, s, &ms, &timed_out);
            if (!rc && !timed_out && ms / steps < best) { best = ms / steps; bc = k; bs = s; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the state as it was (after an error too: the schedule it had), then
    // the choice
    const std::string err = c->err;
    c->parity = parity0;
    c->steps = steps0;
    c->launches = launches0;
    for (int i = 0; i < c->n; ++i)
        CK(c, cudaMemcpy(c->h[i].pop[c->parity], snap[i].data(), snap[i].size(), cudaMemcpyHostToDevice));
    CK(c, cudaMemset(c->d_status, 0, c->n * sizeof(int)));
    if (rc) {
        apply_schedule(c, cfg0, sched0);
        c->err = err;
        return rc;
    }
    if (!(best < 1e300)) {
        apply_schedule(c, cfg0, sched0);
        return fail(c, LBM_ETIMEOUT, "every candidate's bounded device waits gave up%s");
    }
    rc = apply_schedule(c, bc, bs);
    if (rc) return rc;
    if (tile_config) *tile_config = bc;
    if (schedule) *schedule = bs;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

int lbm_use_graphs(lbm_ctx* c, int on) {
    if (!c) return LBM_EINVAL;
    if (on && c->stream == nullptr) return fail(c, LBM_EINVAL, "CUDA graphs need a non-default stream%s");
    c->use_graphs = on != 0;
    if (!on) drop_graphs(c);
    return LBM_OK;
}

int lbm_capture_graphs(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    if (!c->use_graphs || c->sched >= 3) return LBM_OK;
    int rc = ready(c);
    if (rc) return rc;
    CK(c, cudaSetDevice(c->device));
    for (int parity = 0; parity < 2; ++parity)
        for (int level = 0; level < kGraphLevels; ++level)
            if ((rc = ensure_graph(c, parity, level))) return rc;
    return LBM_OK;
}

long long lbm_steps_done(lbm_ctx* c) { return c ? c->steps : -1; }
long long lbm_kernel_launches(lbm_ctx* c) { return c ? c->launches : -1; }

int lbm_bytes_per_update(int precision) {
    const int e = esize(precision);
    return e ? 18 * e : LBM_EINVAL;
}

const char* lbm_last_error(lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
