// batch.cu -- many independent instances of Alg. 1 (FP32 working, n <= 64) in a
// fixed number of launches: the Gram work items and the combine live in
// gram_ozaki.cu; here, one CTA per instance for the n x n stage (Alg. 1 lines
// 3-5, the preconditioned form of Alg. 2 in FP64), and U (line 6) over the row
// tiles of all instances.
//
// n x n stage of one instance (256 threads, M then R in shared memory): a
// pivoted Cholesky P^T M P = R^T R, then a one-sided Jacobi SVD of X = R^T
// whose converged columns y_c give lambda_c = |y_c|^2 and the eigenvectors
// y_c / |y_c| of P^T M P.  Column pairs follow the round-robin tournament
// (n/2 disjoint pairs per round); a group of 8 lanes handles one pair, each
// lane every 8th row.  Rotation (p, q): alpha = |x_p|^2, beta = |x_q|^2,
// gamma = x_p . x_q; skipped when |gamma| <= tol sqrt(alpha beta), otherwise
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = t c, x_p <- c x_p - s x_q, x_q <- s x_p + c x_q,
// alpha <- alpha - t gamma, beta <- beta + t gamma (norms recomputed from the
// columns at the start of every sweep).  The angle and the clear-cut tests are
// evaluated in FP32 (they only set how fast the off-diagonal shrinks); the
// columns, the applied rotation and the borderline tests are FP64.
#include "internal.cuh"

namespace tsvd {
namespace {

constexpr int BT = 256;      // threads per instance CTA
constexpr int BGROUP = 8;    // lanes per column pair

__device__ __forceinline__ unsigned group_mask() { return 0xffu << (threadIdx.x & 24); }
__device__ __forceinline__ double group_sum(double v) {
    const unsigned mask = group_mask();  // the 8 lanes of this group only
#pragma unroll
    for (int o = BGROUP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

__device__ __forceinline__ int player(int pos, int r, int N) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (N - 1); }

// double <-> float by integer bit operations (GB300's FP64 pipe is narrow).  to_f32
// truncates the significand and maps magnitudes outside the normal float range to 0 or
// FLT_MAX: it only feeds angles and tests whose accuracy sets the convergence speed.
__device__ __forceinline__ float to_f32(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned sg = (unsigned)(b >> 63) << 31;
    if (ex < -126) return __uint_as_float(sg);
    if (ex > 127) return __uint_as_float(sg | 0x7f7fffffu);
    return __uint_as_float(sg | ((unsigned)(ex + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}
__device__ __forceinline__ double to_f64(float x) {  // exact for normal floats and zero
    const unsigned b = __float_as_uint(x);
    const unsigned ex = (b >> 23) & 0xff;
    if (ex == 0) return 0.0;
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                            ((unsigned long long)(ex + 896) << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

__global__ void __launch_bounds__(BT) eig_batch_kernel(const BatchInst* __restrict__ inst, double tol,
                                                       int max_sweeps, DevInfo* __restrict__ infos) {
    extern __shared__ double sm[];
    __shared__ double nrm[64];
    __shared__ int perm[64];
    __shared__ int s_piv, s_fail, s_count[2];
    __shared__ unsigned long long s_off;
    const BatchInst& d = inst[blockIdx.x];
    DevInfo* info = infos + blockIdx.x;
    const int n = d.n, LD = n + 1, tid = threadIdx.x;
    const double tol2 = tol * tol;
    const float tol_f = (float)tol;
    double* M = sm;  // [n][LD]: M, then row k = row k of R = column k of X
    for (int idx = tid; idx < n * n; idx += BT) {
        const int i = idx % n, j = idx / n;
        M[i * LD + j] = d.G[i + (size_t)j * n];
    }
    if (tid < n) perm[tid] = tid;
    if (tid == 0) {
        s_fail = 0;
        s_count[0] = s_count[1] = 0;
        s_off = 0ull;
    }
    __syncthreads();

    // ---- pivoted Cholesky in place
    int k = 0;
    for (; k < n; ++k) {
        if (tid < 32) {
            double bv = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const double v = M[i * LD + i];
                if (v > bv) { bv = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (tid == 0) {
                s_piv = bi;
                if (!(bv > 0.0) || !isfinite(bv)) s_fail = 1;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_piv;
        if (p != k) {
            for (int j = tid; j < n; j += BT) {
                const double t = M[k * LD + j]; M[k * LD + j] = M[p * LD + j]; M[p * LD + j] = t;
            }
            __syncthreads();
            for (int i = tid; i < n; i += BT) {
                const double t = M[i * LD + k]; M[i * LD + k] = M[i * LD + p]; M[i * LD + p] = t;
            }
            if (tid == 0) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
            __syncthreads();
        }
        const double rkk = sqrt(M[k * LD + k]);
        const double inv = 1.0 / rkk;
        __syncthreads();
        for (int j = k + 1 + tid; j < n; j += BT) M[k * LD + j] *= inv;
        if (tid == 0) M[k * LD + k] = rkk;
        __syncthreads();
        const int t = n - k - 1;
        for (int idx = tid; idx < t * t; idx += BT) {
            const int i = k + 1 + idx % t, j = k + 1 + idx / t;
            M[i * LD + j] = fma(-M[k * LD + i], M[k * LD + j], M[i * LD + j]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < n * n; idx += BT) {
        const int c = idx / n, r = idx % n;
        if (r < c || c >= k) M[c * LD + r] = 0.0;
    }
    if (tid == 0 && k < n) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
    __syncthreads();

    // ---- one-sided Jacobi on the columns x_c = row c of R
    const int N = (n + 1) & ~1;
    const int grp = tid / BGROUP, gl = tid % BGROUP;
    int sweep = 0;
    bool converged = false;
    while (sweep < max_sweeps) {
        for (int c = grp; c < n; c += BT / BGROUP) {
            double a = 0.0;
            for (int i = gl; i < n; i += BGROUP) a = fma(M[c * LD + i], M[c * LD + i], a);
            a = group_sum(a);
            if (gl == 0) nrm[c] = a;
        }
        if (tid == 0) s_off = 0ull;
        __syncthreads();
        unsigned long long off_bits = 0ull;
        for (int r = 0; r < N - 1; ++r) {
            if (grp < N / 2) {
                int p = player(grp, r, N), q = player(N - 1 - grp, r, N);
                if (p > q) { const int t = p; p = q; q = t; }
                if (q < n) {
                    double* xp = M + p * LD;
                    double* xq = M + q * LD;
                    double g = 0.0;
                    for (int i = gl; i < n; i += BGROUP) g = fma(xp[i], xq[i], g);
                    g = group_sum(g);
                    const double a = nrm[p], b = nrm[q];
                    // the scaled test |g| > tol sqrt(a b): in FP32 when the ratio is clearly on one
                    // side (factor 2), exactly in FP64 otherwise
                    const float af = to_f32(a), bf = to_f32(b), gf = fabsf(to_f32(g));
                    const bool in_range = af > 1e-30f && af < 1e30f && bf > 1e-30f && bf < 1e30f && gf < 1e30f;
                    const float rr = in_range ? gf * rsqrtf(af) * rsqrtf(bf) : 0.0f;
                    bool rot;
                    if (in_range && rr > 2.0f * tol_f) rot = true;
                    else if (in_range && rr < 0.5f * tol_f) rot = false;
                    else rot = g != 0.0 && a > 0.0 && b > 0.0 && g * g > tol2 * (a * b);
                    if (rot) {
                        // Rutishauser's t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / 2g,
                        // in FP32 from ratios <= 1, and c0 = 1 / sqrt(1 + t^2), s0 = t c0; then
                        // (c, s) = (c0, s0) f with f = 1 - e/2 + 3e^2/8, e = c0^2 + s0^2 - 1
                        // (|e| ~ 2^-24): orthogonal to FP64 precision.
                        double c, s, t;
                        if (in_range) {  // then rr > 0: g is a normal float, hf != 0
                            // b - a in FP64 first: for nearly equal norms (clustered sigma) the difference
                            // of two FP32 roundings would be noise and the angle would not shrink g
                            const float df = to_f32(b - a), hf = 2.0f * to_f32(g);
                            const float adf = fabsf(df), ahf = fabsf(hf);
                            const float sz = (df == 0.0f || (df > 0.0f) == (hf > 0.0f)) ? 1.0f : -1.0f;
                            float tf;
                            if (adf >= ahf) {
                                const float z = ahf / adf;
                                tf = sz * z / (1.0f + sqrtf(fmaf(z, z, 1.0f)));
                            } else {
                                const float w = adf / ahf;
                                tf = sz / (w + sqrtf(fmaf(w, w, 1.0f)));
                            }
                            const float cf = rsqrtf(fmaf(tf, tf, 1.0f));
                            const double c0 = to_f64(cf), s0 = to_f64(tf * cf);
                            const double e = fma(c0, c0, fma(s0, s0, -1.0));
                            const double f = fma(e, fma(e, 0.375, -0.5), 1.0);
                            c = c0 * f;
                            s = s0 * f;
                            t = to_f64(tf);
                        } else {  // norms or g outside the float range: the angle in FP64
                            const double zeta = (b - a) / (2.0 * g);
                            const double az = fabs(zeta);
                            t = az > 1e150 ? 0.5 / az : 1.0 / (az + sqrt(fma(az, az, 1.0)));
                            t = copysign(t, zeta);
                            c = 1.0 / sqrt(fma(t, t, 1.0));
                            s = t * c;
                        }
                        for (int i = gl; i < n; i += BGROUP) {
                            const double u = xp[i], v = xq[i];
                            xp[i] = fma(c, u, -s * v);
                            xq[i] = fma(s, u, c * v);
                        }
                        // norms follow a - t g, b + t g; one that dropped 16-fold is recomputed
                        const double tg = t * g;
                        double na = a - tg, nb = b + tg;
                        __syncwarp(group_mask());
                        if (na < 0.0625 * a) {
                            double r = 0.0;
                            for (int i = gl; i < n; i += BGROUP) r = fma(xp[i], xp[i], r);
                            na = group_sum(r);
                        }
                        if (nb < 0.0625 * b) {
                            double r = 0.0;
                            for (int i = gl; i < n; i += BGROUP) r = fma(xq[i], xq[i], r);
                            nb = group_sum(r);
                        }
                        if (gl == 0) {
                            nrm[p] = na;
                            nrm[q] = nb;
                            atomicAdd(&s_count[sweep & 1], 1);
                        }
                    }
                    if (gl == 0 && !rot) off_bits = max(off_bits, (unsigned long long)__float_as_uint(rr));
                }
            }
            __syncthreads();
        }
        if (off_bits) atomicMax(&s_off, off_bits);
        ++sweep;
        const int cnt = s_count[(sweep - 1) & 1];
        __syncthreads();
        if (tid == 0) s_count[(sweep - 1) & 1] = 0;
        if (cnt == 0) {
            converged = true;
            break;
        }
    }

    // ---- lambda_c = |x_c|^2, V (original row order) = x_c / |x_c|
    for (int c = grp; c < n; c += BT / BGROUP) {
        double a = 0.0;
        for (int i = gl; i < n; i += BGROUP) a = fma(M[c * LD + i], M[c * LD + i], a);
        a = group_sum(a);
        const double nc = a > 0.0 ? sqrt(a) : 0.0;
        if (gl == 0) d.lam[c] = a;
        for (int i = gl; i < n; i += BGROUP)
            d.Vh[perm[i] + (size_t)c * n] = nc > 0.0 ? M[c * LD + i] / nc : (perm[i] == c ? 1.0 : 0.0);
    }
    if (tid == 0) {
        info->sweeps = sweep;
        info->off_norm = (double)__uint_as_float((unsigned)s_off);  // largest FP32 ratio left unrotated
        if (!converged) atomicOr(&info->flags, FLAG_NO_CONVERGENCE);
    }
}

// Alg. 1 lines 4-5 per instance: descending order, sign rule (the largest-magnitude
// entry of each column positive, lowest index on ties), sigma = sqrt(lambda), the
// casts to FP32 and W = RN(V / sigma).
__global__ void __launch_bounds__(64) finish_batch_kernel(const BatchInst* __restrict__ inst,
                                                          DevInfo* __restrict__ infos) {
    __shared__ int order[64];
    __shared__ double sig[64], sgn[64];
    const BatchInst& d = inst[blockIdx.x];
    DevInfo* info = infos + blockIdx.x;
    const int n = d.n, tid = threadIdx.x;
    if (tid < n) {
        const double li = d.lam[tid];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = d.lam[j];
            if (lj > li || (lj == li && j < tid)) ++rank;
        }
        order[rank] = tid;
    }
    __syncthreads();
    if (tid < n) {
        const int src = order[tid];
        const double l = d.lam[src];
        if (!(l > 0.0)) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
        sig[tid] = l > 0.0 ? sqrt(l) : 0.0;
        int best = 0;
        double bv = fabs(d.Vh[(size_t)src * n]);
        for (int r = 1; r < n; ++r) {
            const double v = fabs(d.Vh[r + (size_t)src * n]);
            if (v > bv) { bv = v; best = r; }
        }
        sgn[tid] = d.Vh[best + (size_t)src * n] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    if (tid == 0 && n > 1 && sig[n - 1] < 1.1102230246251565e-16 * sig[0]) atomicOr(&info->flags, FLAG_NOT_FULL_RANK);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int r = idx % n, k = idx / n;
        const float vw = (float)(sgn[k] * d.Vh[r + (size_t)order[k] * n]);
        d.V[r + (size_t)k * d.ldv] = vw;
        d.W[r + (size_t)k * n] = vw / (float)sig[k];
    }
    if (tid < n) d.sigma[tid] = (float)sig[tid];
}

// fma.rn.f32x2: two IEEE FP32 FMAs (a row pair of A times a duplicated W entry)
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// U = A W over the row tiles of all instances.  CTA b takes a contiguous range of tiles
// (so W, held duplicated {w, w} in shared memory, is reloaded only when the instance
// changes).  A thread owns 4 rows (two row pairs) by 16 columns; the 256 threads cover
// batch_u_rows(n) rows (more rows when fewer 16-column groups are needed), load four
// columns of A ahead of their FMAs, and accumulate with packed FP32 FMAs (the rounding
// model of eq. (AV-0): each entry is an ordinary FP32 dot product).
__global__ void __launch_bounds__(256, 2) u_batch_kernel(const BatchInst* __restrict__ inst, int count,
                                                         int64_t utiles) {
    __shared__ unsigned long long Ws[64 * 64];
    const int64_t per = (utiles + gridDim.x - 1) / gridDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(utiles, t0 + per);
    if (t0 >= t1) return;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last instance with utile0 <= t0
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].utile0 <= t0) lo = mid; else hi = mid - 1;
    }
    int cur = -1;
    for (int64_t tile = t0; tile < t1; ++tile) {
        while (lo + 1 < count && inst[lo + 1].utile0 <= tile) ++lo;
        const BatchInst& d = inst[lo];
        const int n = d.n;
        if (lo != cur) {
            __syncthreads();  // the previous instance's reads of Ws are done
            for (int idx = threadIdx.x; idx < n * 64; idx += blockDim.x) {
                const int c = idx / 64, k = idx % 64;
                const float w = k < n ? d.W[c + (size_t)k * n] : 0.f;
                Ws[idx] = pack2(w, w);
            }
            __syncthreads();
            cur = lo;
        }
        const int R = batch_u_rows(n) / 256;  // 4, 2 or 1 row groups of 256
        const int rg = threadIdx.x % (64 * R), cg = threadIdx.x / (64 * R);
        const int64_t r0 = (tile - d.utile0) * batch_u_rows(n) + 4 * rg;
        if (cg * 16 >= n || r0 >= d.m) continue;
        const bool full = r0 + 3 < d.m;
        const bool vec = full && ((uintptr_t)d.A % 16 == 0) && (d.lda % 4 == 0) && ((uintptr_t)d.U % 16 == 0) &&
                         (d.ldu % 4 == 0);
        unsigned long long acc[2][16];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[r][k] = 0ull;
        for (int c0 = 0; c0 < n; c0 += 4) {
            unsigned long long a[4][2];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = c0 + cc;
                const float* src = d.A + (size_t)c * d.lda + r0;
                float v[4];
                if (c < n && vec) {
                    const float4 q = __ldcs(reinterpret_cast<const float4*>(src));
                    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[r] = (c < n && r0 + r < d.m) ? src[r] : 0.f;
                }
                a[cc][0] = pack2(v[0], v[1]);
                a[cc][1] = pack2(v[2], v[3]);
            }
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                if (c0 + cc < n) {
                    const unsigned long long* w = Ws + (c0 + cc) * 64 + cg * 16;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const unsigned long long wk = w[k];
                        acc[0][k] = ffma2(a[cc][0], wk, acc[0][k]);
                        acc[1][k] = ffma2(a[cc][1], wk, acc[1][k]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int j = cg * 16 + k;
            if (j < n) {
                float u[4];
                unpack2(acc[0][k], u[0], u[1]);
                unpack2(acc[1][k], u[2], u[3]);
                float* dst = d.U + (size_t)j * d.ldu + r0;
                if (vec) {
                    __stcs(reinterpret_cast<float4*>(dst), make_float4(u[0], u[1], u[2], u[3]));
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r0 + r < d.m) dst[r] = u[r];
                }
            }
        }
    }
}

__global__ void finalize_batch_kernel(DevInfo* __restrict__ infos, int count, DevInfo* agg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int f = infos[i].flags;
        if (f) atomicOr(&agg->flags, f);
        int st = TSVD_OK;
        if (f & FLAG_NONFINITE) st = TSVD_ERR_NONFINITE;
    else if (f & FLAG_BAD_SCALE) st = TSVD_ERR_ARG;
        else if (f & FLAG_TIMEOUT) st = TSVD_ERR_TIMEOUT;
        else if (f & FLAG_NOT_FULL_RANK) st = TSVD_ERR_NOT_FULL_RANK;
        else if (f & FLAG_NO_CONVERGENCE) st = TSVD_ERR_NO_CONVERGENCE;
        infos[i].flags = st;
    }
}

}  // namespace

cudaError_t launch_eig_batch(const BatchInst* inst, int count, double tol, int max_sweeps, DevInfo* infos,
                             cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const size_t smem = sizeof(double) * 64 * 65;
    cudaError_t e = cudaFuncSetAttribute(eig_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    eig_batch_kernel<<<count, BT, smem, s>>>(inst, tol, max_sweeps, infos);
    return cudaGetLastError();
}

cudaError_t launch_finish_batch(const BatchInst* inst, int count, DevInfo* infos, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    finish_batch_kernel<<<count, 64, 0, s>>>(inst, infos);
    return cudaGetLastError();
}

cudaError_t launch_u_batch(const BatchInst* inst, int count, int64_t utiles, int grid, cudaStream_t s) {
    if (count == 0 || utiles == 0) return cudaSuccess;
    const int64_t g = utiles < grid ? utiles : grid;
    u_batch_kernel<<<(unsigned)g, 256, 0, s>>>(inst, count, utiles);
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(DevInfo* infos, int count, DevInfo* agg, cudaStream_t s) {
    if (count > 0) finalize_batch_kernel<<<(count + 255) / 256, 256, 0, s>>>(infos, count, agg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_finalize_info(agg, s);
}

}  // namespace tsvd
