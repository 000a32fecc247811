// The proposal network of the learned MT proposal: a perceptron 16 -> 64 -> 64 -> 16
// with ReLU after the two hidden layers, BF16 weights, inputs and activations and FP32
// accumulation on the fifth-generation tensor cores (tcgen05.mma kind::f16), trained
// on the GPU by its own backward pass and Adam.  The paper has no learned part; the
// network's outputs parameterise a Gaussian proposal of the NCV process noise, whose
// importance weights keep the posterior exact.
//
// One block of 128 threads handles 128 samples (thread = sample = TMEM lane).  Forward:
//   D1 = A0 W1^T, a1 = relu(D1 + b1); D2 = A1 W2^T, a2 = relu(D2 + b2); y = A2 W3^T + b3.
// Training adds, for the loss L = (1/B) sum_i l_i with l_i the Gaussian negative
// log-likelihood of the target t_i (3) under N(mu = y[0:3], diag exp(2 y[3:6])):
//   dy -> dA2 = dy W3, dz2 = dA2 . 1[z2 > 0], dA1 = dz2 W2, dz1 = dA1 . 1[z1 > 0],
//   dW3 = dy^T a2, dW2 = dz2^T a1, dW1 = dz1^T a0 and the bias sums,
// every product on the tensor cores: the data gradients as 128-row tiles, the weight
// gradients as (hidden x samples) tiles padded to 128 rows.  The per-block gradients
// land in a partial buffer that k_mlp_adam reduces in a fixed order before the update.
// dy and dz enter the GEMMs rounded to BF16; the bias sums use them in FP32.
#include <cuda_bf16.h>

#include <string>

#include "bp_handle.cuh"
#include "tc_sm100.cuh"

namespace bp {

constexpr int MLP_IN = 16, MLP_H = 64, MLP_OUT = 16, MLP_TD = 3;
constexpr int MLP_W1 = 0, MLP_B1 = MLP_W1 + MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H, MLP_B2 = MLP_W2 + MLP_H * MLP_H,
              MLP_W3 = MLP_B2 + MLP_H, MLP_B3 = MLP_W3 + MLP_OUT * MLP_H, MLP_NPARAM = MLP_B3 + MLP_OUT;
constexpr int MLP_WAIT = 1 << 20;

// shared-memory tiles (bytes), each a multiple of 128 B
struct MlpSmem {
    int w1, w2, w3, w3t, w2t, a0, a0t, a1, a1t, a2, a2tp, dy, dyt, dz2, dz2tp, dz1tp, red, total;
    __host__ __device__ explicit MlpSmem(bool train) {
        int o = 0;
        auto take = [&](int bytes) { const int r = o; o += bytes; return r; };
        w1 = take(MLP_H * MLP_IN * 2);
        w2 = take(MLP_H * MLP_H * 2);
        w3 = take(MLP_OUT * MLP_H * 2);
        a0 = take(128 * MLP_IN * 2);
        a1 = take(128 * MLP_H * 2);
        a2 = take(128 * MLP_H * 2);
        if (train) {
            w3t = take(MLP_H * MLP_OUT * 2);
            w2t = take(MLP_H * MLP_H * 2);
            a0t = take(MLP_IN * 128 * 2);
            a1t = take(MLP_H * 128 * 2);
            a2tp = take(128 * 128 * 2);
            dy = take(128 * MLP_OUT * 2);
            dyt = take(MLP_OUT * 128 * 2);
            dz2 = take(128 * MLP_H * 2);
            dz2tp = take(128 * 128 * 2);
            dz1tp = take(128 * 128 * 2);
        } else {
            w3t = w2t = a0t = a1t = a2tp = dy = dyt = dz2 = dz2tp = dz1tp = 0;
        }
        red = take(4 * (2 * MLP_H + MLP_OUT + 1) * 4);   // per-warp bias and loss sums
        total = take(64);                                 // mbarrier + TMEM slot
        total = o;
    }
};

__device__ __forceinline__ void st_bf16(char* base, int off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}
// eight consecutive K elements (k % 8 == 0) of one row: one 16-byte store
__device__ __forceinline__ void st_bf16x8(char* base, int off, const float* v) {
    __nv_bfloat162 q[4];
    for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(q);
}

template <bool TRAIN>
__global__ void __launch_bounds__(128) k_mlp(const float* __restrict__ prm, const float* __restrict__ X,
                                             const float* __restrict__ T, int B, float inv_batch,
                                             float* __restrict__ Y, float* __restrict__ gpart,
                                             float* __restrict__ lpart, int* __restrict__ err) {
    extern __shared__ __align__(1024) char smem[];
    const MlpSmem L(TRAIN);
    char* sW1 = smem + L.w1; char* sW2 = smem + L.w2; char* sW3 = smem + L.w3;
    char* sA0 = smem + L.a0; char* sA1 = smem + L.a1; char* sA2 = smem + L.a2;
    float* red = reinterpret_cast<float*>(smem + L.red);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.total - 64);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i = blockIdx.x * 128 + tid;
    const bool act = i < B;
    constexpr uint32_t NCOL = TRAIN ? 512 : 256;
    const uint32_t mb = tc::smem_u32(mbar);
    uint32_t n_commit = 0;
    bool bad = false;
    if (warp == 0) tc::tmem_alloc(tslot, NCOL);
    if (tid == 0) { tc::mbar_init(mb, 1); tc::mbar_init_fence(); }

    // weights (FP32 master -> BF16 tiles; B operands are N x K, K-major)
    for (int t = tid; t < MLP_H * MLP_IN; t += 128) {
        const int o = t / MLP_IN, k = t % MLP_IN;
        st_bf16(sW1, tc::core_off16(o, k, MLP_IN), prm[MLP_W1 + t]);
    }
    for (int t = tid; t < MLP_H * MLP_H; t += 128) {
        const int o = t / MLP_H, k = t % MLP_H;
        st_bf16(sW2, tc::core_off16(o, k, MLP_H), prm[MLP_W2 + t]);
        if (TRAIN) st_bf16(smem + L.w2t, tc::core_off16(k, o, MLP_H), prm[MLP_W2 + t]);   // W2^T: (in, out)
    }
    for (int t = tid; t < MLP_OUT * MLP_H; t += 128) {
        const int o = t / MLP_H, k = t % MLP_H;
        st_bf16(sW3, tc::core_off16(o, k, MLP_H), prm[MLP_W3 + t]);
        if (TRAIN) st_bf16(smem + L.w3t, tc::core_off16(k, o, MLP_OUT), prm[MLP_W3 + t]);  // W3^T: (in, out)
    }
    // this thread's input row (zeros past the batch)
    {
        float x[MLP_IN];
        for (int k = 0; k < MLP_IN; ++k) x[k] = act ? X[(size_t)i * MLP_IN + k] : 0.f;
        st_bf16x8(sA0, tc::core_off16(tid, 0, MLP_IN), x);
        st_bf16x8(sA0, tc::core_off16(tid, 8, MLP_IN), x + 8);
        if (TRAIN)
            for (int k = 0; k < MLP_IN; ++k) st_bf16(smem + L.a0t, tc::core_off16(k, tid, 128), x[k]);
    }
    if (TRAIN) {   // rows 64..127 of the padded (hidden x samples) tiles stay zero
        for (int t = tid; t < 128 * 128 * 2 / 2 / 16; t += 128) {
            const uint4 zz = make_uint4(0, 0, 0, 0);
            reinterpret_cast<uint4*>(smem + L.a2tp + 128 * 128)[t] = zz;
            reinterpret_cast<uint4*>(smem + L.dz2tp + 128 * 128)[t] = zz;
            reinterpret_cast<uint4*>(smem + L.dz1tp + 128 * 128)[t] = zz;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);

    // D[dcol..] (+)= A (128 x K) B^T (N x K), K in steps of 16
    auto gemm = [&](uint32_t dcol, const char* A, const char* Bm, int N, int K) {
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        const uint32_t a = tc::smem_u32(A), b = tc::smem_u32(Bm);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint32_t o = (uint32_t)ks * 256u;
            tc::mma_bf16(tmem + dcol, tc::smem_desc(a + o, 128, sbo), tc::smem_desc(b + o, 128, sbo),
                         tc::idesc_bf16_f32(128, N), ks > 0);
        }
    };
    // operands written by all threads -> visible to the tensor cores; thread 0 issues
    // the GEMMs of this stage and commits; every thread waits (bounded)
    auto stage = [&](auto&& issue) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !bad) { issue(); tc::mma_commit(mb); }
        ++n_commit;
        if (!bad && !tc::mbar_wait(mb, (n_commit - 1) & 1u, MLP_WAIT)) bad = true;
        tc::fence_after_sync();
    };
    auto ld64 = [&](uint32_t col, float* v) {
        uint32_t r[32];
        tc::tmem_ld32(tlane + col, r); tc::tmem_ld_wait();
        for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
        tc::tmem_ld32(tlane + col + 32, r); tc::tmem_ld_wait();
        for (int c = 0; c < 32; ++c) v[32 + c] = __uint_as_float(r[c]);
    };
    auto ld16 = [&](uint32_t col, float* v) {
        uint32_t r[16];
        tc::tmem_ld16(tlane + col, r); tc::tmem_ld_wait();
        for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
    };
    // deterministic block sum of n per-thread values (n <= 64) into red[.. n]
    auto block_sum = [&](const float* v, int n, float* out_g) {
        __syncthreads();
        for (int c = 0; c < n; ++c) {
            const float w = warp_sum_f(v[c]);
            if (lane == 0) red[warp * 64 + c] = w;
        }
        __syncthreads();
        if (tid < n) out_g[tid] = ((red[tid] + red[64 + tid]) + red[128 + tid]) + red[192 + tid];
        __syncthreads();
    };

    // ---- forward
    stage([&] { gemm(0, sA0, sW1, MLP_H, MLP_IN); });
    uint64_t m1 = 0, m2 = 0;
    float v[64];
    ld64(0, v);
    for (int c = 0; c < MLP_H; ++c) {
        const float z = v[c] + prm[MLP_B1 + c];
        if (z > 0.f) m1 |= 1ull << c;
        v[c] = fmaxf(z, 0.f);
    }
    for (int k = 0; k < MLP_H; k += 8) st_bf16x8(sA1, tc::core_off16(tid, k, MLP_H), v + k);
    if (TRAIN)
        for (int k = 0; k < MLP_H; ++k) st_bf16(smem + L.a1t, tc::core_off16(k, tid, 128), v[k]);
    stage([&] { gemm(64, sA1, sW2, MLP_H, MLP_H); });
    ld64(64, v);
    for (int c = 0; c < MLP_H; ++c) {
        const float z = v[c] + prm[MLP_B2 + c];
        if (z > 0.f) m2 |= 1ull << c;
        v[c] = fmaxf(z, 0.f);
    }
    for (int k = 0; k < MLP_H; k += 8) st_bf16x8(sA2, tc::core_off16(tid, k, MLP_H), v + k);
    if (TRAIN)
        for (int k = 0; k < MLP_H; ++k) st_bf16(smem + L.a2tp, tc::core_off16(k, tid, 128), v[k]);
    stage([&] { gemm(128, sA2, sW3, MLP_OUT, MLP_H); });
    float y[MLP_OUT];
    ld16(128, y);
    for (int c = 0; c < MLP_OUT; ++c) y[c] += prm[MLP_B3 + c];
    if (!TRAIN) {
        if (act)
            for (int c = 0; c < MLP_OUT; ++c) Y[(size_t)i * MLP_OUT + c] = y[c];
    } else {
        // ---- loss and dy
        float dy[MLP_OUT], loss = 0.f;
        for (int c = 0; c < MLP_OUT; ++c) dy[c] = 0.f;
        if (act) {
            for (int a = 0; a < MLP_TD; ++a) {
                const float mu = y[a], ls = y[MLP_TD + a];
                const float e = expf(-2.f * ls), d = T[(size_t)i * MLP_TD + a] - mu;
                loss += 0.5f * d * d * e + ls;
                dy[a] = -d * e * inv_batch;
                dy[MLP_TD + a] = (1.f - d * d * e) * inv_batch;
            }
        }
        st_bf16x8(smem + L.dy, tc::core_off16(tid, 0, MLP_OUT), dy);
        st_bf16x8(smem + L.dy, tc::core_off16(tid, 8, MLP_OUT), dy + 8);
        for (int c = 0; c < MLP_OUT; ++c) st_bf16(smem + L.dyt, tc::core_off16(c, tid, 128), dy[c]);
        float* gp = gpart + (size_t)blockIdx.x * MLP_NPARAM;
        block_sum(dy, MLP_OUT, gp + MLP_B3);
        {
            float lv[1] = {loss};
            block_sum(lv, 1, lpart + blockIdx.x);
        }
        // ---- dA2 = dy W3 (cols 144..207), dW3^T = a2^T dy (cols 208..223)
        stage([&] {
            gemm(144, smem + L.dy, smem + L.w3t, MLP_H, MLP_OUT);
            gemm(208, smem + L.a2tp, smem + L.dyt, MLP_OUT, 128);
        });
        ld64(144, v);
        for (int c = 0; c < MLP_H; ++c) v[c] = ((m2 >> c) & 1ull) ? v[c] : 0.f;
        for (int k = 0; k < MLP_H; k += 8) st_bf16x8(smem + L.dz2, tc::core_off16(tid, k, MLP_H), v + k);
        for (int k = 0; k < MLP_H; ++k) st_bf16(smem + L.dz2tp, tc::core_off16(k, tid, 128), v[k]);
        block_sum(v, MLP_H, gp + MLP_B2);
        if (warp < 2) {   // rows 0..63: hidden unit h = tid
            float g[MLP_OUT];
            ld16(208, g);
            for (int c = 0; c < MLP_OUT; ++c) gp[MLP_W3 + c * MLP_H + tid] = g[c];
        }
        // ---- dA1 = dz2 W2 (cols 224..287), dW2 = dz2^T a1 (cols 288..351)
        stage([&] {
            gemm(224, smem + L.dz2, smem + L.w2t, MLP_H, MLP_H);
            gemm(288, smem + L.dz2tp, smem + L.a1t, MLP_H, 128);
        });
        ld64(224, v);
        for (int c = 0; c < MLP_H; ++c) v[c] = ((m1 >> c) & 1ull) ? v[c] : 0.f;
        for (int k = 0; k < MLP_H; ++k) st_bf16(smem + L.dz1tp, tc::core_off16(k, tid, 128), v[k]);
        block_sum(v, MLP_H, gp + MLP_B1);
        if (warp < 2) {
            float g[64];
            ld64(288, g);
            for (int n = 0; n < MLP_H; ++n) gp[MLP_W2 + tid * MLP_H + n] = g[n];
        }
        // ---- dW1 = dz1^T a0 (cols 352..367)
        stage([&] { gemm(352, smem + L.dz1tp, smem + L.a0t, MLP_IN, 128); });
        if (warp < 2) {
            float g[MLP_IN];
            ld16(352, g);
            for (int k = 0; k < MLP_IN; ++k) gp[MLP_W1 + tid * MLP_IN + k] = g[k];
        }
    }
    if (bad && lane == 0) atomicOr(err, 1);
    if (tid == 0 && n_commit > 0) tc::mbar_wait(mb, (n_commit - 1) & 1u, MLP_WAIT);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

// fixed-order sum of the per-block gradients; then (adam) one Adam step on the FP32
// master parameters, or (grads) the summed gradients written out
__global__ void k_mlp_adam(int nblk, const float* __restrict__ gpart, const float* __restrict__ lpart,
                           float* __restrict__ prm, float* __restrict__ m, float* __restrict__ v, int t, float lr,
                           float b1, float b2, float eps, int apply, float* __restrict__ gout,
                           float* __restrict__ loss) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0 && loss) {
        double l = 0.0;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = (float)l;
    }
    if (j >= MLP_NPARAM) return;
    double g = 0.0;
    for (int b = 0; b < nblk; ++b) g += gpart[(size_t)b * MLP_NPARAM + j];
    if (gout) gout[j] = (float)g;
    if (!apply) return;
    const float gf = (float)g;
    const float mj = b1 * m[j] + (1.f - b1) * gf;
    const float vj = b2 * v[j] + (1.f - b2) * gf * gf;
    m[j] = mj;
    v[j] = vj;
    const float mh = mj / (1.f - powf(b1, (float)t)), vh = vj / (1.f - powf(b2, (float)t));
    prm[j] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace bp

using namespace bp;

struct bp_mlp {
    float* prm = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* gpart = nullptr;
    float* lpart = nullptr;
    int* err = nullptr;
    int cap_blocks = 0;
    int t = 0;
    cudaStream_t st = nullptr;
    std::string msg;
};

static bp_status mlp_fail(bp_mlp* h, bp_status s, const char* what) {
    if (h) h->msg = what;
    return s;
}

static bool mlp_reserve(bp_mlp* h, int nblk) {
    if (nblk <= h->cap_blocks) return true;
    cudaFree(h->gpart);
    cudaFree(h->lpart);
    h->gpart = nullptr;
    h->lpart = nullptr;
    if (cudaMalloc(&h->gpart, (size_t)nblk * MLP_NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->lpart, (size_t)nblk * sizeof(float)) != cudaSuccess)
        return false;
    h->cap_blocks = nblk;
    return true;
}

static bp_status mlp_check_err(bp_mlp* h) {
    int e = 0;
    if (cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return mlp_fail(h, BP_ERR_CUDA, "CUDA error");
    if (e) return mlp_fail(h, BP_ERR_TIMEOUT, "tensor-core wait timed out");
    return BP_OK;
}

// forward (train = false) or forward + backward into the partial buffers
static bp_status mlp_launch(bp_mlp* h, bool train, const float* X, const float* T, int B, float* Y) {
    const int nblk = (B + 127) / 128;
    const MlpSmem L(train);
    if ((size_t)L.total > (size_t)smem_optin()) return mlp_fail(h, BP_ERR_CAPACITY, "shared memory");
    if (train) {
        if (!mlp_reserve(h, nblk)) return mlp_fail(h, BP_ERR_CUDA, "allocation failed");
        smem_allow_max((const void*)k_mlp<true>);
        k_mlp<true><<<nblk, 128, L.total, h->st>>>(h->prm, X, T, B, 1.f / (float)B, nullptr, h->gpart, h->lpart, h->err);
    } else {
        smem_allow_max((const void*)k_mlp<false>);
        k_mlp<false><<<nblk, 128, L.total, h->st>>>(h->prm, X, nullptr, B, 0.f, Y, nullptr, nullptr, h->err);
    }
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(h, BP_ERR_CUDA, "launch failed");
    return BP_OK;
}

void mlp_forward_async(const bp_mlp* net, const float* X, int B, float* Y, cudaStream_t st) {
    if (B < 1) return;
    const MlpSmem L(false);
    smem_allow_max((const void*)k_mlp<false>);
    k_mlp<false><<<(B + 127) / 128, 128, L.total, st>>>(net->prm, X, nullptr, B, 0.f, Y, nullptr, nullptr, net->err);
}

extern "C" {

bp_status bp_mlp_create(const float* params_host, void* cuda_stream, bp_mlp** out) {
    if (!params_host || !out) return BP_ERR_INVALID_ARG;
    *out = nullptr;
    bp_mlp* h = new bp_mlp();
    h->st = static_cast<cudaStream_t>(cuda_stream);
    const size_t pb = (size_t)MLP_NPARAM * sizeof(float);
    if (cudaMalloc(&h->prm, pb) != cudaSuccess || cudaMalloc(&h->m, pb) != cudaSuccess ||
        cudaMalloc(&h->v, pb) != cudaSuccess || cudaMalloc(&h->err, sizeof(int)) != cudaSuccess ||
        cudaMemcpyAsync(h->prm, params_host, pb, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
        cudaMemsetAsync(h->m, 0, pb, h->st) != cudaSuccess || cudaMemsetAsync(h->v, 0, pb, h->st) != cudaSuccess ||
        cudaMemsetAsync(h->err, 0, sizeof(int), h->st) != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) {
        bp_mlp_free(h);
        return BP_ERR_CUDA;
    }
    *out = h;
    return BP_OK;
}

bp_status bp_mlp_get_params(bp_mlp* h, float* params_host) {
    if (!h || !params_host) return BP_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(params_host, h->prm, (size_t)MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, h->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return mlp_fail(h, BP_ERR_CUDA, "CUDA error");
    return BP_OK;
}

bp_status bp_mlp_forward(bp_mlp* h, const float* X_dev, int B, float* Y_dev) {
    if (!h || B < 0 || (B > 0 && (!X_dev || !Y_dev))) return BP_ERR_INVALID_ARG;
    if (B == 0) return BP_OK;
    const bp_status s = mlp_launch(h, false, X_dev, nullptr, B, Y_dev);
    if (s != BP_OK) return s;
    return mlp_check_err(h);
}

bp_status bp_mlp_grads(bp_mlp* h, const float* X_dev, const float* T_dev, int B, float* grad_dev, float* loss_dev) {
    if (!h || B < 1 || !X_dev || !T_dev || !grad_dev) return BP_ERR_INVALID_ARG;
    bp_status s = mlp_launch(h, true, X_dev, T_dev, B, nullptr);
    if (s != BP_OK) return s;
    const int nblk = (B + 127) / 128;
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, h->st>>>(nblk, h->gpart, h->lpart, h->prm, h->m, h->v, 1, 0.f, 0.f,
                                                            0.f, 0.f, 0, grad_dev, loss_dev);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(h, BP_ERR_CUDA, "launch failed");
    return mlp_check_err(h);
}

bp_status bp_mlp_train_step(bp_mlp* h, const float* X_dev, const float* T_dev, int B, float lr, float* loss_dev) {
    if (!h || B < 1 || !X_dev || !T_dev || !(lr >= 0.f)) return BP_ERR_INVALID_ARG;
    bp_status s = mlp_launch(h, true, X_dev, T_dev, B, nullptr);
    if (s != BP_OK) return s;
    const int nblk = (B + 127) / 128;
    h->t += 1;
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, h->st>>>(nblk, h->gpart, h->lpart, h->prm, h->m, h->v, h->t, lr,
                                                            0.9f, 0.999f, 1e-8f, 1, nullptr, loss_dev);
    if (cudaGetLastError() != cudaSuccess) return mlp_fail(h, BP_ERR_CUDA, "launch failed");
    return BP_OK;
}

bp_status bp_mlp_sync(bp_mlp* h) {
    if (!h) return BP_ERR_INVALID_ARG;
    return mlp_check_err(h);
}

bp_status bp_mlp_free(bp_mlp* h) {
    if (!h) return BP_OK;
    cudaFree(h->prm);
    cudaFree(h->m);
    cudaFree(h->v);
    cudaFree(h->gpart);
    cudaFree(h->lpart);
    cudaFree(h->err);
    delete h;
    return BP_OK;
}

const char* bp_mlp_last_error(const bp_mlp* h) { return h ? h->msg.c_str() : ""; }

}  // extern "C"
