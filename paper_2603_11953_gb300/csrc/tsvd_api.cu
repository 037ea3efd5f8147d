// tsvd_api.cu -- the C ABI (include/tsvd.h): argument checks, workspace,
// and the launch sequence of Algorithm 1 on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "internal.cuh"

using namespace tsvd;

// the autotuner's choice for one shape (opts.autotune)
struct TuneChoice {
    int split_k;    // Gram CTAs (0: one per SM)
    int u_variant;  // 0 tensor-core U, 1 CUDA-core U
    float gram_ms;  // the chosen Gram's time
    float u_ms;     // the chosen U's time (0: U not tuned)
};

struct tsvd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    tsvd_opts opts{};
    int sm_count = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    DevInfo* dinfo = nullptr;
    // per-stage events of the last `timing` calls (a ring of 4 events per call)
    std::vector<cudaEvent_t> ev;
    long long calls = 0;     // timed calls so far
    bool have_times = false;
    // pinned staging of the batched descriptors (reused once its last copy is done)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;
    // second stream for small kernels that run beside the main sequence (the kappa(B) estimate)
    EigSide side{nullptr, nullptr, nullptr};
    // autotuner choices by (m, n, working, TMA-loadable input)
    std::map<std::tuple<long long, int, int, int>, TuneChoice> tuned;
};

namespace {

constexpr double U_FP64 = 1.1102230246251565e-16;  // 2^-53

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

tsvd_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TSVD_OK;
    if (e == cudaErrorNotSupported) return TSVD_ERR_UNSUPPORTED;
    if (e == cudaErrorMemoryAllocation) return TSVD_ERR_ALLOC;
    return TSVD_ERR_CUDA;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

tsvd_status ensure_ws(tsvd_ctx* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return TSVD_OK;
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TSVD_ERR_ALLOC;
    }
    h->ws_bytes = bytes;
    return TSVD_OK;
}

size_t wsize(int working) { return working == 0 ? sizeof(float) : sizeof(double); }

// Workspace carve-up of one solve: [partials][G][G_lo][lam][Vh][scratch 2n^2][W].
struct Layout {
    size_t part = 0, G = 0, Glo = 0, lam = 0, Vh = 0, scratch = 0, W = 0, total = 0;
};
Layout layout_for(int64_t n, size_t part_bytes, int working) {
    Layout L;
    size_t off = 0;
    L.part = off; off += align_up(part_bytes);
    L.G = off; off += align_up(sizeof(double) * n * n);
    L.Glo = off; off += align_up(sizeof(double) * n * n);
    L.lam = off; off += align_up(sizeof(double) * n);
    L.Vh = off; off += align_up(sizeof(double) * n * n);
    L.scratch = off; off += align_up(sizeof(double) * (3 * n * n + n));  // X, perm, Cholesky scratch (n > 64)
    L.W = off; off += align_up(wsize(working) * n * n);
    L.total = off;
    return L;
}

char* base(tsvd_ctx* h) { return static_cast<char*>(h->ws); }

bool valid_prec_pair(tsvd_prec working, tsvd_prec higher) {
    return (working == TSVD_FP32 || working == TSVD_FP64) && (higher == TSVD_FP64 || higher == TSVD_DD);
}

// tcgen05 Gram (default) when the input allows TMA; gram_variant 2 forces the
// mma.sync version of the same Ozaki arithmetic.
bool use_tc(tsvd_ctx* h, const void* A, int working, int n, int64_t lda) {
    return h->opts.gram_variant == 0 && gram_tc_ok(A, working, n, lda);
}

// FP64 working precision on the tensor cores: exact 23-bit pieces of the
// column-scaled A, the Gram of the needed 32-column block pairs of the piece
// matrix X into the double-double G3, then the piece sums into G (and G_lo).
bool use_fp64_pieces(tsvd_ctx* h, int working, int64_t n) {
    return working == TSVD_FP64 && h->opts.gram_variant == 0 && n <= 64;
}

// Fixed column scales (tsvd_opts.fixed_scale, and the row-sharded entry points): FP32,
// n <= 64, TMA-loadable input.
tsvd_status fixed_scale_check(const void* A, int working, int64_t n, int64_t lda) {
    if (working != TSVD_FP32 || n > 64) return TSVD_ERR_UNSUPPORTED;
    if (!gram_tc_ok(A, working, (int)n, lda)) return TSVD_ERR_ALIGN;
    return TSVD_OK;
}
constexpr size_t FIXED_EXTRA = 512;  // column maxima (n unsigned) and exponents (n int) after the partials

tsvd_status run_gram_fp64(tsvd_ctx* h, const void* A, int64_t m, int n, int64_t lda, double* G, double* G_lo,
                          int64_t ldg, size_t part_off) {
    GramPlan plan = gram_tc_plan(m, 64, h->sm_count, h->opts.split_k);
    plan.wait_cycles = h->opts.timeout_cycles;
    char* part = base(h) + part_off;
    void* extra = part + align_up(gram_partials_bytes(plan));
    cudaError_t e = launch_fp64_split(static_cast<const double*>(A), m, n, lda, extra, h->dinfo, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    const float* X = fp64_split_matrix(extra);
    const int C = 4 * fp64_block_cols(n);
    const int64_t ldx = fp64_split_ld(m);
    double* g3lo = nullptr;
    double* g3 = fp64_g3(extra, m, n, &g3lo);
    const int nb = C / 32;
    bool diag_done[8] = {false, false, false, false, false, false, false, false};
    for (int b1 = 0; b1 < nb - 1; ++b1)
        for (int b2 = b1 + 1; b2 < nb; ++b2) {
            if (!fp64_pair_needed(n, b1, b2)) continue;
            int wmask = 4;
            if (!diag_done[b1] && fp64_pair_needed(n, b1, b1)) { wmask |= 1; diag_done[b1] = true; }
            if (!diag_done[b2] && fp64_pair_needed(n, b2, b2)) { wmask |= 2; diag_done[b2] = true; }
            e = launch_gram_tc2(X, m, C, ldx, 32 * b1, 32 * b2, plan, part, h->dinfo, h->stream);
            if (e == cudaSuccess)
                e = launch_gram_combine2(plan, part, C, 32 * b1, 32 * b2, wmask, g3, g3lo, C, h->stream);
            if (e != cudaSuccess) return from_cuda(e);
        }
    return from_cuda(launch_fp64_fold(extra, m, n, G, G_lo, ldg, h->stream));
}

// Gram into G (and G_lo) for one matrix.  Caller validated the arguments.
tsvd_status run_gram(tsvd_ctx* h, const void* A, int64_t m, int n, int64_t lda, int working,
                     double* G, double* G_lo, int64_t ldg, size_t part_off) {
    cudaError_t e;
    if (h->opts.gram_variant == 1) {
        e = launch_gram_plain(A, working, m, n, lda, h->sm_count, base(h) + part_off, G, ldg, h->dinfo,
                              h->stream);
        if (e == cudaSuccess && G_lo) e = cudaMemsetAsync(G_lo, 0, sizeof(double) * ldg * n, h->stream);
        return from_cuda(e);
    }
    if (use_fp64_pieces(h, working, n)) return run_gram_fp64(h, A, m, n, lda, G, G_lo, ldg, part_off);
    if (h->opts.fixed_scale) {
        // every column's exponent over the whole of A first, then the Gram on those fixed scales
        GramPlan plan = gram_tc_plan(m, n, h->sm_count, h->opts.split_k);
        plan.wait_cycles = h->opts.timeout_cycles;
        char* ex = base(h) + part_off + align_up(gram_partials_bytes(plan));
        int* E = reinterpret_cast<int*>(ex + 256);
        e = launch_colexp(static_cast<const float*>(A), m, n, lda, reinterpret_cast<unsigned*>(ex), E, h->dinfo,
                          h->sm_count, h->stream);
        if (e != cudaSuccess) return from_cuda(e);
        plan.E_fixed = E;
        e = launch_gram_tc(A, m, n, lda, plan, base(h) + part_off, h->dinfo, h->stream);
        if (e != cudaSuccess) return from_cuda(e);
        return from_cuda(launch_gram_combine(plan, base(h) + part_off, n, G, G_lo, ldg, h->stream));
    }
    const bool tc = use_tc(h, A, working, n, lda);
    if (tc && n > 64) {
        // 32-column blocks b1 < b2, one launch per pair: the cross tile always, block b1's
        // diagonal tile from the pair (b1, b1 + 1), the last block's from (nb - 2, nb - 1)
        GramPlan plan = gram_tc_plan(m, 64, h->sm_count, h->opts.split_k);
        plan.wait_cycles = h->opts.timeout_cycles;
        const int nb = (n + 31) / 32;
        for (int b1 = 0; b1 < nb - 1; ++b1)
            for (int b2 = b1 + 1; b2 < nb; ++b2) {
                const int wmask = 4 | (b2 == b1 + 1 ? 1 : 0) | (b1 == nb - 2 && b2 == nb - 1 ? 2 : 0);
                e = launch_gram_tc2(A, m, n, lda, 32 * b1, 32 * b2, plan, base(h) + part_off, h->dinfo, h->stream);
                if (e == cudaSuccess)
                    e = launch_gram_combine2(plan, base(h) + part_off, n, 32 * b1, 32 * b2, wmask, G, G_lo, ldg,
                                             h->stream);
                if (e != cudaSuccess) return from_cuda(e);
            }
        return TSVD_OK;
    }
    GramPlan plan = tc ? gram_tc_plan(m, n, h->sm_count, h->opts.split_k)
                       : gram_plan(m, n, h->sm_count, h->opts.split_k);
    plan.wait_cycles = h->opts.timeout_cycles;
    e = tc ? launch_gram_tc(A, m, n, lda, plan, base(h) + part_off, h->dinfo, h->stream)
           : launch_gram_ozaki(A, working, m, n, lda, plan, base(h) + part_off, h->dinfo, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(launch_gram_combine(plan, base(h) + part_off, n, G, G_lo, ldg, h->stream));
}

size_t part_bytes_for(tsvd_ctx* h, const void* A, int working, int64_t m, int n, int64_t lda) {
    if (h->opts.gram_variant == 1) return gram_plain_partials_bytes(m, n, h->sm_count);
    if (use_fp64_pieces(h, working, n))
        return align_up(gram_partials_bytes(gram_tc_plan(m, 64, h->sm_count, h->opts.split_k))) +
               fp64_extra_bytes(m, n);
    if (h->opts.fixed_scale)
        return align_up(gram_partials_bytes(gram_tc_plan(m, n, h->sm_count, h->opts.split_k))) + FIXED_EXTRA;
    if (use_tc(h, A, working, n, lda)) return gram_partials_bytes(gram_tc_plan(m, n, h->sm_count, h->opts.split_k));
    return gram_partials_bytes(gram_plan(m, n, h->sm_count, h->opts.split_k));
}

bool gram_supported(tsvd_ctx* h, const void* A, int working, int64_t n, int64_t lda) {
    if (working == TSVD_FP64) return h->opts.gram_variant == 1 ? n <= 64 : use_fp64_pieces(h, working, n);
    if (n <= 64) return true;
    // 64 < n <= 256: the tensor-core Gram over pairs of 32-column blocks
    return n <= 256 && use_tc(h, A, working, (int)n, lda);
}

double jacobi_tol(tsvd_ctx* h, int64_t n) {
    return h->opts.jacobi_tol > 0.0 ? h->opts.jacobi_tol : (double)n * U_FP64;
}
constexpr double U_DD = 4.930380657631324e-32;  // 2^-104
double jacobi_tol_dd(tsvd_ctx* h, int64_t n) {
    return h->opts.jacobi_tol > 0.0 ? h->opts.jacobi_tol : (double)n * U_DD;
}
int max_sweeps(tsvd_ctx* h) { return h->opts.max_sweeps > 0 ? h->opts.max_sweeps : 40; }

// The eigen stage on M (n x n, ldm): unsorted lambda and V into lam / Vh.
cudaError_t run_eig(tsvd_ctx* h, const double* M, int n, int64_t ldm, double* scratch, double* lam,
                    double* Vh) {
    if (h->opts.eig_variant == EIG_ALG2) {
        // Algorithm 2: the SVD of R runs at the working precision; its skip threshold is
        // n 2^-24 (the rounding level of an FP32 dot product) unless jacobi_tol is given
        const float tol = h->opts.jacobi_tol > 0.0 ? (float)h->opts.jacobi_tol : (float)n * 5.9604644775390625e-8f;
        return launch_eig_alg2(M, n, ldm, tol, max_sweeps(h), scratch, lam, Vh, h->dinfo, h->stream);
    }
    const bool one_sided = n <= 256 && (h->opts.eig_variant == EIG_ONE_SIDED || h->opts.eig_variant == EIG_DEFAULT);
    if (one_sided)
        return launch_eig_onesided(M, n, ldm, jacobi_tol(h, n), max_sweeps(h), scratch, lam, Vh, h->dinfo,
                                   h->stream, &h->side, h->opts.timeout_cycles);
    return launch_jacobi(M, n, ldm, jacobi_tol(h, n), max_sweeps(h), scratch, lam, Vh, h->dinfo, h->stream);
}

// ---------------------------------------------------------------- autotuner (opts.autotune = 1)
// The first tsvd_gram or tsvd_solve of a shape (m, n, working precision, TMA-loadable input) on a
// handle times the Gram with the candidate split-K CTA counts (one per SM, half, twice, three
// times that) and, when the call asks for an FP32 U of n <= 64 that both U kernels accept, the
// tensor-core and the CUDA-core U; each candidate runs three times (the first untimed) into the
// handle's workspace, and the fastest are kept for the handle's later calls of that shape.
// This synchronises the stream once per shape; while the stream is being captured, or when the
// caller fixed split_k or u_variant, the defaults apply.
float time_once(tsvd_ctx* h, cudaEvent_t e0, cudaEvent_t e1, const std::function<cudaError_t()>& run) {
    float best = -1.0f;
    for (int rep = 0; rep < 3; ++rep) {
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) return -1.0f;
        if (run() != cudaSuccess) return -1.0f;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.0f;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
        if (rep > 0 && (best < 0.0f || ms < best)) best = ms;
    }
    return best;
}

const TuneChoice* autotune(tsvd_ctx* h, const void* A, int64_t m, int n, int64_t lda, int working, void* U,
                           int64_t ldu) {
    if (!h->opts.autotune || h->opts.gram_variant != 0 || h->opts.fixed_scale || h->opts.split_k > 0) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return nullptr;
    }
    const int tc = use_tc(h, A, working, n, lda) ? 1 : 0;
    const auto key = std::make_tuple((long long)m, n, working, tc);
    const auto it = h->tuned.find(key);
    if (it != h->tuned.end()) return &it->second;
    const int cand[4] = {0, h->sm_count / 2, 2 * h->sm_count, 3 * h->sm_count};
    size_t need = 0;
    for (int c : cand) {
        h->opts.split_k = c;
        need = std::max(need, layout_for(n, part_bytes_for(h, A, working, m, n, lda), working).total);
    }
    h->opts.split_k = 0;
    if (ensure_ws(h, need) != TSVD_OK) return nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return nullptr;
    }
    TuneChoice ch{0, 0, -1.0f, 0.0f};
    for (int c : cand) {
        h->opts.split_k = c;
        const Layout L = layout_for(n, part_bytes_for(h, A, working, m, n, lda), working);
        double* G = reinterpret_cast<double*>(base(h) + L.G);
        double* G_lo = working == TSVD_FP64 ? reinterpret_cast<double*>(base(h) + L.Glo) : nullptr;
        const float ms = time_once(h, e0, e1, [&]() {
            const tsvd_status st = run_gram(h, A, m, n, lda, working, G, G_lo, n, L.part);
            return st == TSVD_OK ? cudaSuccess : cudaErrorUnknown;
        });
        if (ms > 0.0f && (ch.gram_ms < 0.0f || ms < ch.gram_ms)) { ch.gram_ms = ms; ch.split_k = c; }
    }
    h->opts.split_k = 0;
    if (U && working == TSVD_FP32 && h->opts.u_variant == 0 && compute_u_tc_ok(A, working, m, n, lda) &&
        compute_u_v2_ok(A, working, m, n, lda, U, ldu)) {
        const Layout L = layout_for(n, part_bytes_for(h, A, working, m, n, lda), working);
        const float* W = reinterpret_cast<const float*>(base(h) + L.W);
        const float t_tc = time_once(h, e0, e1, [&]() {
            return launch_compute_u_tc(static_cast<const float*>(A), m, n, lda, W, static_cast<float*>(U), ldu,
                                       h->sm_count, h->dinfo, h->stream);
        });
        const float t_cc = time_once(h, e0, e1, [&]() {
            return launch_compute_u_v2(static_cast<const float*>(A), m, n, lda, W, static_cast<float*>(U), ldu,
                                       h->sm_count, h->dinfo, h->stream);
        });
        if (t_tc > 0.0f && t_cc > 0.0f) {
            ch.u_variant = t_cc < t_tc ? 1 : 0;
            ch.u_ms = t_cc < t_tc ? t_cc : t_tc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    if (ch.gram_ms < 0.0f) return nullptr;
    return &(h->tuned[key] = ch);
}

// the tuned options for one call, put back when it returns
struct TunedOpts {
    tsvd_ctx* h;
    int split_k, u_variant;
    TunedOpts(tsvd_ctx* hh, const TuneChoice* c) : h(hh), split_k(hh->opts.split_k), u_variant(hh->opts.u_variant) {
        if (c) {
            h->opts.split_k = c->split_k;
            h->opts.u_variant = c->u_variant;
        }
    }
    ~TunedOpts() {
        h->opts.split_k = split_k;
        h->opts.u_variant = u_variant;
    }
};

int ring(const tsvd_ctx* h) { return (int)(h->ev.size() / 4); }
void record(tsvd_ctx* h, int k) {
    if (h->opts.timing) cudaEventRecord(h->ev[4 * (size_t)(h->calls % ring(h)) + k], h->stream);
}

// One instance of Algorithm 1, workspace already sized by the caller.
tsvd_status solve_one(tsvd_ctx* h, const void* A, int64_t m, int n, int64_t lda, int working, int higher,
                      void* sigma, void* V, int64_t ldv, void* U, int64_t ldu, tsvd_info* info,
                      bool timed) {
    const Layout L = layout_for(n, part_bytes_for(h, A, working, m, n, lda), working);
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double* G = reinterpret_cast<double*>(base(h) + L.G);
    double* lam = reinterpret_cast<double*>(base(h) + L.lam);
    double* Vh = reinterpret_cast<double*>(base(h) + L.Vh);
    double* scratch = reinterpret_cast<double*>(base(h) + L.scratch);
    void* W = base(h) + L.W;
    if (timed) record(h, 0);
    // double-double n x n stage: FP64 working with the double-double Gram
    const bool dd_eig = higher == TSVD_DD && use_fp64_pieces(h, working, n);
    double* G_lo = dd_eig ? reinterpret_cast<double*>(base(h) + L.Glo) : nullptr;
    tsvd_status st = run_gram(h, A, m, n, lda, working, G, G_lo, n, L.part);
    if (st != TSVD_OK) return st;
    if (timed) record(h, 1);
    e = dd_eig ? launch_eig_dd(G, G_lo, n, n, jacobi_tol_dd(h, n), max_sweeps(h), lam, Vh, h->dinfo, h->stream)
               : run_eig(h, G, n, n, scratch, lam, Vh);
    if (e != cudaSuccess) return from_cuda(e);
    e = launch_finish(lam, Vh, n, working, sigma, V, ldv, W, nullptr, nullptr, 0, h->dinfo, h->stream,
                      dd_eig ? U_DD : U_FP64);
    if (e != cudaSuccess) return from_cuda(e);
    if (timed) record(h, 2);
    if (U) {
        if (h->opts.u_variant == 0 && compute_u_tc_ok(A, working, m, n, lda))
            e = launch_compute_u_tc(static_cast<const float*>(A), m, n, lda, static_cast<const float*>(W),
                                    static_cast<float*>(U), ldu, h->sm_count, h->dinfo, h->stream);
        else if (compute_u_v2_ok(A, working, m, n, lda, U, ldu))
            e = launch_compute_u_v2(static_cast<const float*>(A), m, n, lda, static_cast<const float*>(W),
                                    static_cast<float*>(U), ldu, h->sm_count, h->dinfo, h->stream);
        else
            e = launch_compute_u(A, working, m, n, lda, W, U, ldu, h->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (timed) record(h, 3);
    e = launch_finalize_info(h->dinfo, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (info) {
        e = cudaMemcpyAsync(info, h->dinfo, sizeof(DevInfo), cudaMemcpyDefault, h->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (timed) {
        h->have_times = true;
        ++h->calls;
    }
    return TSVD_OK;
}

}  // namespace

extern "C" {

const char* tsvd_status_string(tsvd_status s) {
    switch (s) {
        case TSVD_OK: return "TSVD_OK";
        case TSVD_ERR_ARG: return "TSVD_ERR_ARG";
        case TSVD_ERR_ALIGN: return "TSVD_ERR_ALIGN";
        case TSVD_ERR_NONFINITE: return "TSVD_ERR_NONFINITE";
        case TSVD_ERR_NOT_FULL_RANK: return "TSVD_ERR_NOT_FULL_RANK";
        case TSVD_ERR_NO_CONVERGENCE: return "TSVD_ERR_NO_CONVERGENCE";
        case TSVD_ERR_TIMEOUT: return "TSVD_ERR_TIMEOUT";
        case TSVD_ERR_UNSUPPORTED: return "TSVD_ERR_UNSUPPORTED";
        case TSVD_ERR_CUDA: return "TSVD_ERR_CUDA";
        case TSVD_ERR_ALLOC: return "TSVD_ERR_ALLOC";
    }
    return "TSVD_ERR_UNKNOWN";
}

tsvd_status tsvd_create(tsvd_handle* out, int device, void* stream, const tsvd_opts* opts) {
    if (!out) return TSVD_ERR_ARG;
    *out = nullptr;
    if (opts) {
        if (opts->slices != 0 && opts->slices != GRAM_DIGITS) return TSVD_ERR_UNSUPPORTED;
        if (opts->chunk_rows != 0 && opts->chunk_rows != GRAM_KC) return TSVD_ERR_UNSUPPORTED;
        if (opts->split_k < 0 || opts->max_sweeps < 0 || opts->jacobi_tol < 0.0) return TSVD_ERR_ARG;
        if (opts->eig_variant < 0 || opts->eig_variant > 3) return TSVD_ERR_UNSUPPORTED;
        if (opts->gram_variant < 0 || opts->gram_variant > 2) return TSVD_ERR_ARG;
        if (opts->u_variant < 0 || opts->u_variant > 1) return TSVD_ERR_ARG;
        if (opts->timing < 0 || opts->timeout_cycles < 0) return TSVD_ERR_ARG;
        if (opts->fixed_scale < 0 || opts->fixed_scale > 1) return TSVD_ERR_ARG;
        if (opts->fixed_scale && opts->gram_variant != 0) return TSVD_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return TSVD_ERR_CUDA;
    }
    DeviceGuard g(device);
    tsvd_ctx* h = new (std::nothrow) tsvd_ctx();
    if (!h) return TSVD_ERR_ALLOC;
    h->device = device;
    h->stream = static_cast<cudaStream_t>(stream);
    if (opts) h->opts = *opts;
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&h->dinfo, sizeof(DevInfo)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return TSVD_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&h->side.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (h->side.stream) cudaStreamDestroy(h->side.stream);
        if (h->side.fork) cudaEventDestroy(h->side.fork);
        cudaFree(h->dinfo);
        delete h;
        return TSVD_ERR_CUDA;
    }
    if (h->opts.timing > 0) {
        h->ev.assign(4 * (size_t)(h->opts.timing < TSVD_MAX_TIMED ? h->opts.timing : TSVD_MAX_TIMED), nullptr);
        for (auto& ev : h->ev) cudaEventCreate(&ev);
    }
    *out = h;
    return TSVD_OK;
}

tsvd_status tsvd_destroy(tsvd_handle h) {
    if (!h) return TSVD_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->dinfo) cudaFree(h->dinfo);
    for (auto& ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    if (h->stage) cudaFreeHost(h->stage);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    if (h->side.stream) cudaStreamSynchronize(h->side.stream), cudaStreamDestroy(h->side.stream);
    if (h->side.fork) cudaEventDestroy(h->side.fork);
    if (h->side.join) cudaEventDestroy(h->side.join);
    delete h;
    return TSVD_OK;
}

tsvd_status tsvd_gram(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                      tsvd_prec working, tsvd_prec higher, double* G, int64_t ldg) {
    if (!h || !A || !G || m < 1 || n < 1 || lda < m || ldg < n || !valid_prec_pair(working, higher))
        return TSVD_ERR_ARG;
    if (!gram_supported(h, A, working, n, lda)) return TSVD_ERR_UNSUPPORTED;
    if (higher == TSVD_DD && h->opts.gram_variant == 1) return TSVD_ERR_UNSUPPORTED;
    if (h->opts.fixed_scale) {
        const tsvd_status fs = fixed_scale_check(A, working, n, lda);
        if (fs != TSVD_OK) return fs;
    }
    DeviceGuard g(h->device);
    const TunedOpts tuned(h, autotune(h, A, m, (int)n, lda, working, nullptr, 0));
    const size_t pb = part_bytes_for(h, A, working, m, (int)n, lda);
    tsvd_status st = ensure_ws(h, align_up(pb));
    if (st != TSVD_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double* G_lo = higher == TSVD_DD ? G + ldg * n : nullptr;
    st = run_gram(h, A, m, (int)n, lda, working, G, G_lo, ldg, 0);
    if (st != TSVD_OK) return st;
    return from_cuda(launch_finalize_info(h->dinfo, h->stream));
}

tsvd_status tsvd_eig(tsvd_handle h, const double* M, int64_t n, int64_t ldm, double* lambda,
                     double* V, int64_t ldv, tsvd_info* info) {
    if (!h || !M || !lambda || !V || n < 1 || ldm < n || ldv < n) return TSVD_ERR_ARG;
    if (n > 256 || (h->opts.eig_variant == EIG_ALG2 && n > 64)) return TSVD_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    const Layout L = layout_for(n, 0, 1);
    tsvd_status st = ensure_ws(h, L.total);
    if (st != TSVD_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double* lam = reinterpret_cast<double*>(base(h) + L.lam);
    double* Vh = reinterpret_cast<double*>(base(h) + L.Vh);
    double* scratch = reinterpret_cast<double*>(base(h) + L.scratch);
    e = run_eig(h, M, (int)n, ldm, scratch, lam, Vh);
    if (e == cudaSuccess)
        e = launch_finish(lam, Vh, (int)n, 1, nullptr, nullptr, 0, nullptr, lambda, V, ldv, h->dinfo,
                          h->stream);
    if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
    if (e == cudaSuccess && info)
        e = cudaMemcpyAsync(info, h->dinfo, sizeof(DevInfo), cudaMemcpyDefault, h->stream);
    return from_cuda(e);
}

tsvd_status tsvd_solve(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                       tsvd_prec working, tsvd_prec higher, void* sigma, void* V, int64_t ldv,
                       void* U, int64_t ldu, tsvd_info* info) {
    if (!h || !A || !sigma || !V || n < 1 || m < n || lda < m || ldv < n || (U && ldu < m) ||
        !valid_prec_pair(working, higher))
        return TSVD_ERR_ARG;
    // FP32 working: FP64 n x n stage.  FP64 working: double-double Gram, then a
    // double-double (higher = DD) or FP64 (higher = FP64) n x n stage; the plain
    // FP64 Gram (gram_variant 1) has no double-double form.
    if (working == TSVD_FP32 && higher != TSVD_FP64) return TSVD_ERR_UNSUPPORTED;
    // Algorithm 2 (SVD of the cast Cholesky factor at the working precision): FP32 working, n <= 64
    if (h->opts.eig_variant == EIG_ALG2 && (working != TSVD_FP32 || n > 64)) return TSVD_ERR_UNSUPPORTED;
    if (higher == TSVD_DD && h->opts.gram_variant == 1) return TSVD_ERR_UNSUPPORTED;
    if (!gram_supported(h, A, working, n, lda)) return TSVD_ERR_UNSUPPORTED;
    if (h->opts.fixed_scale) {
        const tsvd_status fs = fixed_scale_check(A, working, n, lda);
        if (fs != TSVD_OK) return fs;
    }
    DeviceGuard g(h->device);
    const TunedOpts tuned(h, autotune(h, A, m, (int)n, lda, working, U, ldu));
    const Layout L = layout_for(n, part_bytes_for(h, A, working, m, (int)n, lda), working);
    tsvd_status st = ensure_ws(h, L.total);
    if (st != TSVD_OK) return st;
    h->have_times = false;
    return solve_one(h, A, m, (int)n, lda, working, higher, sigma, V, ldv, U, ldu, info, true);
}

tsvd_status tsvd_autotune_choice(tsvd_handle h, int64_t m, int64_t n, tsvd_prec working, int32_t* split_k,
                                 int32_t* u_variant, float* gram_ms, float* u_ms) {
    if (!h || !split_k) return TSVD_ERR_ARG;
    for (int tc = 1; tc >= 0; --tc) {
        const auto it = h->tuned.find(std::make_tuple((long long)m, (int)n, (int)working, tc));
        if (it == h->tuned.end()) continue;
        *split_k = it->second.split_k;
        if (u_variant) *u_variant = it->second.u_variant;
        if (gram_ms) *gram_ms = it->second.gram_ms;
        if (u_ms) *u_ms = it->second.u_ms;
        return TSVD_OK;
    }
    return TSVD_ERR_ARG;
}

}  // extern "C"

namespace {

// Batched Algorithm 1 (FP32 working, n <= 64): Gram work items (instance, row range of at
// most BATCH_ROWS) in one launch per padded width, one combine launch, one CTA per
// instance for the n x n stage and the finish, U over all instances' row tiles, and
// the statuses: at most nine launches whatever the count.
tsvd_status batch_run(tsvd_ctx* h, int32_t count, const void* const* A, const int64_t* m, const int64_t* n,
                      const int64_t* lda, void* const* sigma, void* const* V, const int64_t* ldv, void* const* U,
                      const int64_t* ldu, tsvd_info* info) {
    std::vector<BatchInst> inst((size_t)count);
    std::vector<BatchGramItem> cls[4];
    std::vector<TcBatchItem> tci;  // tensor-core items (tmap filled in once the offsets are known)
    std::vector<int> tcmap((size_t)count, -1);
    int ntc = 0;
    int slots = 0;
    int64_t utiles = 0;
    size_t per_off = 0;
    std::vector<size_t> per((size_t)count);
    bool vec[4] = {true, true, true, true};
    for (int32_t i = 0; i < count; ++i) {
        BatchInst& d = inst[(size_t)i];
        const int ni = (int)n[i];
        d.A = static_cast<const float*>(A[i]);
        d.m = m[i];
        d.lda = lda[i];
        d.n = ni;
        // the tensor-core Gram where the instance can be TMA-loaded (gram_variant 2 forces the
        // CUDA-core Ozaki kernel); its partials are 64 x 64
        const bool tc = h->opts.gram_variant == 0 && gram_tc_batch_ok(A[i], lda[i]);
        d.NP = tc ? 64 : ni <= 16 ? 16 : ni <= 32 ? 32 : ni <= 48 ? 48 : 64;
        const int c = d.NP / 16 - 1;
        if (!tc && ((uintptr_t)A[i] % 16 != 0 || lda[i] % 4 != 0)) vec[c] = false;
        // n <= 32: two 64-row blocks side by side per tensor-core step (two maps, 32-column boxes)
        const bool pack = tc && ni <= 32 && m[i] >= 128;
        if (tc) tcmap[(size_t)i] = ntc++;
        if (pack) ++ntc;
        d.halves = pack ? 2 : 1;
        d.slot0 = slots;
        d.nslots = (int)((m[i] + BATCH_ROWS - 1) / BATCH_ROWS);
        for (int k = 0; k < d.nslots; ++k) {
            const int64_t r0 = (int64_t)k * BATCH_ROWS;
            const int64_t r1 = std::min<int64_t>(m[i], r0 + BATCH_ROWS);
            if (tc) tci.push_back(TcBatchItem{nullptr, pack ? A[i] : nullptr, r0, r1, ni, slots + k, i, 0});
            else cls[c].push_back(BatchGramItem{i, slots + k, r0, r1});
        }
        slots += d.nslots;
        d.sigma = static_cast<float*>(sigma[i]);
        d.V = static_cast<float*>(V[i]);
        d.ldv = ldv[i];
        const bool want_u = U && U[i];
        d.U = want_u ? static_cast<float*>(U[i]) : nullptr;
        d.ldu = want_u ? ldu[i] : 0;
        d.utile0 = utiles;
        if (want_u) utiles += (m[i] + batch_u_rows(ni) - 1) / batch_u_rows(ni);
        per[(size_t)i] = per_off;
        per_off += align_up(sizeof(double) * (2 * (size_t)ni * ni + ni) + sizeof(float) * (size_t)ni * ni);
    }
    // longest row ranges first within each width (the CTAs take items in order)
    size_t nitems = 0, coff[4];
    for (int c = 0; c < 4; ++c) {
        std::stable_sort(cls[c].begin(), cls[c].end(),
                         [](const BatchGramItem& a, const BatchGramItem& b) { return a.r1 - a.r0 > b.r1 - b.r0; });
        coff[c] = nitems;
        nitems += cls[c].size();
    }
    std::stable_sort(tci.begin(), tci.end(),
                     [](const TcBatchItem& a, const TcBatchItem& b) { return a.r1 - a.r0 > b.r1 - b.r0; });
    // workspace: [descriptors][items][tensor-core items][tensor maps][infos][partials]
    //            [per-instance G, lam, Vh, W]; the first four come through the staging buffer
    const size_t b_inst = align_up(sizeof(BatchInst) * (size_t)count);
    const size_t b_items = align_up(sizeof(BatchGramItem) * nitems);
    const size_t b_tci = align_up(sizeof(TcBatchItem) * tci.size());
    const size_t b_maps = align_up(tc_tmap_bytes() * (size_t)ntc);
    const size_t b_info = align_up(sizeof(DevInfo) * (size_t)count);
    const size_t b_part = align_up(gram_batch_partials_bytes(slots));
    const size_t o_items = b_inst, o_tci = o_items + b_items, o_maps = o_tci + b_tci, o_info = o_maps + b_maps;
    const size_t o_part = o_info + b_info, o_per = o_part + b_part;
    tsvd_status st = ensure_ws(h, o_per + per_off);
    if (st != TSVD_OK) return st;
    for (int32_t i = 0; i < count; ++i) {
        BatchInst& d = inst[(size_t)i];
        char* b = base(h) + o_per + per[(size_t)i];
        const size_t nn = (size_t)d.n * d.n;
        d.G = reinterpret_cast<double*>(b);
        d.lam = d.G + nn;
        d.Vh = d.lam + d.n;
        d.W = reinterpret_cast<float*>(d.Vh + nn);
    }
    // descriptors and items through the pinned staging buffer
    const size_t stage_need = o_info;
    if (h->stage_ev) {
        if (cudaEventSynchronize(h->stage_ev) != cudaSuccess) return from_cuda(cudaGetLastError());
    } else if (cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming) != cudaSuccess) {
        return from_cuda(cudaGetLastError());
    }
    if (h->stage_bytes < stage_need) {
        if (h->stage) cudaFreeHost(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        if (cudaMallocHost(&h->stage, stage_need) != cudaSuccess) {
            cudaGetLastError();
            return TSVD_ERR_ALLOC;
        }
        h->stage_bytes = stage_need;
    }
    char* sb = static_cast<char*>(h->stage);
    std::memcpy(sb, inst.data(), sizeof(BatchInst) * (size_t)count);
    for (int c = 0; c < 4; ++c)
        if (!cls[c].empty())
            std::memcpy(sb + b_inst + sizeof(BatchGramItem) * coff[c], cls[c].data(),
                        sizeof(BatchGramItem) * cls[c].size());
    for (int32_t i = 0; i < count; ++i) {
        const int k = tcmap[(size_t)i];
        if (k < 0) continue;
        const float* Ai = static_cast<const float*>(A[i]);
        const bool pack = inst[(size_t)i].halves == 2;
        cudaError_t em = make_tc_batch_tmap(sb + o_maps + tc_tmap_bytes() * (size_t)k, Ai, m[i], (int)n[i], lda[i],
                                            pack ? 32 : (int)n[i]);
        if (em == cudaSuccess && pack)  // rows 64.. of the same instance
            em = make_tc_batch_tmap(sb + o_maps + tc_tmap_bytes() * (size_t)(k + 1), Ai + 64, m[i] - 64, (int)n[i],
                                    lda[i], 32);
        if (em != cudaSuccess) return TSVD_ERR_UNSUPPORTED;
    }
    for (auto& it : tci) {
        const size_t k = (size_t)tcmap[(size_t)it.inst];
        it.tmap = base(h) + o_maps + tc_tmap_bytes() * k;
        it.tmap2 = it.tmap2 != nullptr ? base(h) + o_maps + tc_tmap_bytes() * (k + 1) : nullptr;
    }
    if (!tci.empty()) std::memcpy(sb + o_tci, tci.data(), sizeof(TcBatchItem) * tci.size());
    cudaError_t e = cudaMemcpyAsync(base(h), sb, stage_need, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->stage_ev, h->stream);
    const BatchInst* dinst = reinterpret_cast<const BatchInst*>(base(h));
    const BatchGramItem* ditems = reinterpret_cast<const BatchGramItem*>(base(h) + o_items);
    DevInfo* dinfos = reinterpret_cast<DevInfo*>(base(h) + o_info);
    void* part = base(h) + o_part;
    if (e == cudaSuccess) e = cudaMemsetAsync(dinfos, 0, sizeof(DevInfo) * (size_t)count, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    record(h, 0);
    e = launch_gram_tc_batch(reinterpret_cast<const TcBatchItem*>(base(h) + o_tci), (int)tci.size(), part, slots,
                             dinfos, h->stream, h->opts.timeout_cycles);
    if (e != cudaSuccess) return from_cuda(e);
    for (int c = 0; c < 4; ++c) {
        e = launch_gram_batch(dinst, ditems + coff[c], (int)cls[c].size(), 16 * (c + 1), vec[c], part, slots, dinfos,
                              h->sm_count, h->stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    e = launch_gram_combine_batch(dinst, count, part, slots, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    record(h, 1);
    e = launch_eig_batch(dinst, count, jacobi_tol(h, 64), max_sweeps(h), dinfos, h->stream);
    if (e == cudaSuccess) e = launch_finish_batch(dinst, count, dinfos, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    record(h, 2);
    e = launch_u_batch(dinst, count, utiles, 16 * h->sm_count, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    record(h, 3);
    e = launch_finalize_batch(dinfos, count, h->dinfo, h->stream);
    if (e == cudaSuccess && info)
        e = cudaMemcpyAsync(info, dinfos, sizeof(DevInfo) * (size_t)count, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (h->opts.timing) {
        h->have_times = true;
        ++h->calls;
    }
    return TSVD_OK;
}

}  // namespace

extern "C" {

tsvd_status tsvd_batch_solve(tsvd_handle h, int32_t count, const void* const* A, const int64_t* m,
                             const int64_t* n, const int64_t* lda, tsvd_prec working,
                             tsvd_prec higher, void* const* sigma, void* const* V,
                             const int64_t* ldv, void* const* U, const int64_t* ldu,
                             tsvd_info* info) {
    if (!h || count < 0 || (count > 0 && (!A || !m || !n || !lda || !sigma || !V || !ldv)))
        return TSVD_ERR_ARG;
    if (!valid_prec_pair(working, higher)) return TSVD_ERR_ARG;
    if (!(working == TSVD_FP32 && higher == TSVD_FP64)) return TSVD_ERR_UNSUPPORTED;
    if (h->opts.fixed_scale) return TSVD_ERR_UNSUPPORTED;
    size_t need = 0;
    for (int32_t i = 0; i < count; ++i) {
        const bool want_u = U && U[i];
        if (!A[i] || !sigma[i] || !V[i] || n[i] < 1 || m[i] < n[i] || lda[i] < m[i] || ldv[i] < n[i] ||
            (want_u && (!ldu || ldu[i] < m[i])))
            return TSVD_ERR_ARG;
        if (n[i] > 64) return TSVD_ERR_UNSUPPORTED;
        need = std::max(need, layout_for(n[i], part_bytes_for(h, A[i], working, m[i], (int)n[i], lda[i]), working).total);
    }
    DeviceGuard g(h->device);
    h->have_times = false;
    if (count == 0) return TSVD_OK;
    if (h->opts.gram_variant != 1) return batch_run(h, count, A, m, n, lda, sigma, V, ldv, U, ldu, info);
    // the plain FP64 comparison form: one instance per launch sequence
    tsvd_status st = ensure_ws(h, need);
    if (st != TSVD_OK) return st;
    for (int32_t i = 0; i < count; ++i) {
        const bool want_u = U && U[i];
        st = solve_one(h, A[i], m[i], (int)n[i], lda[i], working, higher, sigma[i], V[i], ldv[i],
                       want_u ? U[i] : nullptr, want_u ? ldu[i] : 0, info ? info + i : nullptr, false);
        if (st != TSVD_OK) return st;
    }
    return TSVD_OK;
}

tsvd_status tsvd_sync_status(tsvd_handle h) {
    if (!h) return TSVD_ERR_ARG;
    DeviceGuard g(h->device);
    DevInfo d;
    if (cudaMemcpyAsync(&d, h->dinfo, sizeof(d), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return TSVD_ERR_CUDA;
    }
    // Before finalize the word holds flag bits; after it holds a status code.
    return static_cast<tsvd_status>(d.flags);
}

static bool stage_times(tsvd_ctx* h, long long call, float ms[4]) {
    const cudaEvent_t* e = &h->ev[4 * (size_t)(call % ring(h))];
    if (cudaEventSynchronize(e[3]) != cudaSuccess) return false;
    float a = 0, b = 0, c = 0, t = 0;
    cudaEventElapsedTime(&a, e[0], e[1]);
    cudaEventElapsedTime(&b, e[1], e[2]);
    cudaEventElapsedTime(&c, e[2], e[3]);
    cudaEventElapsedTime(&t, e[0], e[3]);
    ms[0] = a; ms[1] = b; ms[2] = c; ms[3] = t;
    return true;
}

tsvd_status tsvd_last_stage_ms(tsvd_handle h, float ms[4]) {
    if (!h || !ms) return TSVD_ERR_ARG;
    if (!h->opts.timing || !h->have_times) return TSVD_ERR_ARG;
    DeviceGuard g(h->device);
    return stage_times(h, h->calls - 1, ms) ? TSVD_OK : TSVD_ERR_CUDA;
}

tsvd_status tsvd_stage_ms_mean(tsvd_handle h, int last, float ms[4]) {
    if (!h || !ms || last < 1) return TSVD_ERR_ARG;
    if (!h->opts.timing || !h->have_times || last > ring(h) || last > h->calls) return TSVD_ERR_ARG;
    DeviceGuard g(h->device);
    double acc[4] = {0, 0, 0, 0};
    for (long long c = h->calls - last; c < h->calls; ++c) {
        float one[4];
        if (!stage_times(h, c, one)) return TSVD_ERR_CUDA;
        for (int k = 0; k < 4; ++k) acc[k] += one[k];
    }
    for (int k = 0; k < 4; ++k) ms[k] = (float)(acc[k] / last);
    return TSVD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- row-sharded Gram (Sec. 4.2.1)
extern "C" {

tsvd_status tsvd_gram_colexp(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda, tsvd_prec working,
                             int32_t* E) {
    if (!h || !A || !E || m < 0 || n < 1 || lda < (m > 1 ? m : 1) || (working != TSVD_FP32 && working != TSVD_FP64))
        return TSVD_ERR_ARG;
    if (working != TSVD_FP32 || n > 64) return TSVD_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    tsvd_status st = ensure_ws(h, 256);
    if (st != TSVD_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e == cudaSuccess)
        e = launch_colexp(static_cast<const float*>(A), m, (int)n, lda, reinterpret_cast<unsigned*>(h->ws), E,
                          h->dinfo, h->sm_count, h->stream);
    if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
    return from_cuda(e);
}

tsvd_status tsvd_gram_partial(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda, tsvd_prec working,
                              const int32_t* E, int64_t* limbs) {
    if (!h || !A || !E || !limbs || m < 0 || n < 1 || lda < (m > 1 ? m : 1) ||
        (working != TSVD_FP32 && working != TSVD_FP64))
        return TSVD_ERR_ARG;
    const tsvd_status fs = fixed_scale_check(A, working, n, lda);
    if (fs != TSVD_OK) return fs;
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (m == 0) {  // a rank without rows contributes zero
        e = cudaMemsetAsync(limbs, 0, sizeof(int64_t) * 4 * (size_t)n * n, h->stream);
        if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
        return from_cuda(e);
    }
    GramPlan plan = gram_tc_plan(m, (int)n, h->sm_count, h->opts.split_k);
    plan.wait_cycles = h->opts.timeout_cycles;
    plan.E_fixed = E;
    tsvd_status st = ensure_ws(h, align_up(gram_partials_bytes(plan)));
    if (st != TSVD_OK) return st;
    e = launch_gram_tc(A, m, (int)n, lda, plan, h->ws, h->dinfo, h->stream);
    if (e == cudaSuccess) e = launch_gram_limbs(plan, h->ws, (int)n, E, reinterpret_cast<long long*>(limbs), h->stream);
    if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
    return from_cuda(e);
}

tsvd_status tsvd_gram_finish(tsvd_handle h, const int64_t* limbs, const int32_t* E, int64_t n, tsvd_prec higher,
                             double* G, int64_t ldg) {
    if (!h || !limbs || !E || !G || n < 1 || ldg < n || (higher != TSVD_FP64 && higher != TSVD_DD))
        return TSVD_ERR_ARG;
    if (n > 64) return TSVD_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    return from_cuda(launch_gram_finish(reinterpret_cast<const long long*>(limbs), (int)n, E, G,
                                        higher == TSVD_DD ? G + ldg * n : nullptr, ldg, h->stream));
}

tsvd_status tsvd_solve_gram(tsvd_handle h, const double* G, int64_t ldg, const void* A, int64_t m, int64_t n,
                            int64_t lda, tsvd_prec working, tsvd_prec higher, void* sigma, void* V, int64_t ldv,
                            void* U, int64_t ldu, tsvd_info* info) {
    if (!h || !G || !sigma || !V || n < 1 || ldg < n || m < 0 || ldv < n || (U && (!A || ldu < (m > 1 ? m : 1))) ||
        (A && lda < (m > 1 ? m : 1)) || !valid_prec_pair(working, higher))
        return TSVD_ERR_ARG;
    if (working != TSVD_FP32 || higher != TSVD_FP64 || n > 256) return TSVD_ERR_UNSUPPORTED;
    if (h->opts.eig_variant == EIG_ALG2 && n > 64) return TSVD_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    const Layout L = layout_for(n, 0, working);
    tsvd_status st = ensure_ws(h, L.total);
    if (st != TSVD_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double* lam = reinterpret_cast<double*>(base(h) + L.lam);
    double* Vh = reinterpret_cast<double*>(base(h) + L.Vh);
    double* scratch = reinterpret_cast<double*>(base(h) + L.scratch);
    void* W = base(h) + L.W;
    // stage events as tsvd_solve records them; the Gram stage is empty here (the caller formed G)
    record(h, 0);
    record(h, 1);
    e = run_eig(h, G, (int)n, ldg, scratch, lam, Vh);
    if (e == cudaSuccess)
        e = launch_finish(lam, Vh, (int)n, working, sigma, V, ldv, W, nullptr, nullptr, 0, h->dinfo, h->stream, U_FP64);
    if (e == cudaSuccess) record(h, 2);
    if (e == cudaSuccess && U && m > 0) {
        if (h->opts.u_variant == 0 && compute_u_tc_ok(A, working, m, (int)n, lda))
            e = launch_compute_u_tc(static_cast<const float*>(A), m, (int)n, lda, static_cast<const float*>(W),
                                    static_cast<float*>(U), ldu, h->sm_count, h->dinfo, h->stream);
        else if (compute_u_v2_ok(A, working, m, (int)n, lda, U, ldu))
            e = launch_compute_u_v2(static_cast<const float*>(A), m, (int)n, lda, static_cast<const float*>(W),
                                    static_cast<float*>(U), ldu, h->sm_count, h->dinfo, h->stream);
        else
            e = launch_compute_u(A, working, m, (int)n, lda, W, U, ldu, h->stream);
    }
    if (e == cudaSuccess && h->opts.timing) {
        record(h, 3);
        h->have_times = true;
        ++h->calls;
    }
    if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, h->dinfo, sizeof(DevInfo), cudaMemcpyDefault, h->stream);
    return from_cuda(e);
}

}  // extern "C"

// ---------------------------------------------------------------- mixed precision Cholesky QR (Sec. 3.1)
extern "C" tsvd_status tsvd_cholqr(tsvd_handle h, const void* A, int64_t m, int64_t n, int64_t lda,
                                   tsvd_prec working, tsvd_prec higher, void* Q, int64_t ldq, double* R,
                                   int64_t ldr, tsvd_info* info) {
    if (!h || !A || n < 1 || m < n || lda < m || (Q && ldq < m) || (R && ldr < n) || !valid_prec_pair(working, higher))
        return TSVD_ERR_ARG;
    if (working != TSVD_FP32 || higher != TSVD_FP64 || n > 64) return TSVD_ERR_UNSUPPORTED;
    if (h->opts.fixed_scale) {
        const tsvd_status fs = fixed_scale_check(A, working, n, lda);
        if (fs != TSVD_OK) return fs;
    }
    DeviceGuard g(h->device);
    const Layout L = layout_for(n, part_bytes_for(h, A, working, m, (int)n, lda), working);
    tsvd_status st = ensure_ws(h, L.total);
    if (st != TSVD_OK) return st;
    cudaError_t e = cudaMemsetAsync(h->dinfo, 0, sizeof(DevInfo), h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    double* G = reinterpret_cast<double*>(base(h) + L.G);
    double* X = reinterpret_cast<double*>(base(h) + L.scratch);
    int* perm = reinterpret_cast<int*>(base(h) + L.scratch + sizeof(double) * (size_t)n * n);
    st = run_gram(h, A, m, (int)n, lda, working, G, nullptr, n, L.part);
    if (st != TSVD_OK) return st;
    e = launch_cholesky(G, (int)n, n, X, perm, h->dinfo, false, h->stream);
    if (e == cudaSuccess)
        e = launch_cholqr_q(static_cast<const float*>(A), m, (int)n, lda, X, static_cast<float*>(Q), ldq, R, ldr,
                            h->sm_count, h->stream);
    if (e == cudaSuccess) e = launch_finalize_info(h->dinfo, h->stream);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, h->dinfo, sizeof(DevInfo), cudaMemcpyDefault, h->stream);
    return from_cuda(e);
}
