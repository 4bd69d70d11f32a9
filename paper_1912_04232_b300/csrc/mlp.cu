// mlp.cu -- the per-atom network of the learned potential (Sec. 4.1):
//   x = (G - mu) / sd,  a1 = W1 x + b1,  h1 = silu(a1),  a2 = W2 h1 + b2,
//   h2 = silu(a2),  E_i = w3 . h2 + b3      (16 -> 64 -> 64 -> 1)
//
// k_mlp_infer : E_i and dE_i/dG_i (backward to the input), one warp per
//               atom, lanes own hidden units (h = lane, lane + 32); FP32
//               on CUDA cores, weights staged in shared memory.
// k_mlp_train : per atom, for the training objective
//                  J = c_E E_i - c_F phi_i,  phi_i = dE_i/dG_i . v_i
//               (v_i = descriptor Jacobian applied to the force error, so
//               sum over atoms of phi carries the force-loss term): forward,
//               tangent along v/sd, and reverse through both -- the
//               "double backward" of the force loss.  Writes the per-atom
//               factors whose outer products sum to the weight gradients.
// k_mlp_grads : the sums over atoms (fixed order, FP64 accumulation).
// k_adam      : Adam on the FP32 parameter vector.
#include "bp.cuh"
#include "common.cuh"

namespace jmd {

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

struct Silu3 {
    float v, d1, d2;   // silu, silu', silu''
};

__device__ __forceinline__ Silu3 silu3(float x)
{
    float s = sigm(x);
    Silu3 r;
    r.v = x * s;
    r.d1 = s * (1.0f + x * (1.0f - s));
    r.d2 = s * (1.0f - s) * (2.0f + x * (1.0f - 2.0f * s));
    return r;
}

// shared-memory copy of the network: W1 [64][16], W2 [64][64] and its
// transpose, biases, w3, b3, normalisation
struct MlpSmem {
    float W1[BP_H * BP_D];
    float W2[BP_H * BP_H];
    float W2T[BP_H * BP_H];
    float b1[BP_H], b2[BP_H], w3[BP_H];
    float mu[BP_D], sd[BP_D];
    float b3;
};

__device__ void stage_params(MlpSmem &S, const float *P, const float *norm)
{
    for (int k = threadIdx.x; k < BP_H * BP_D; k += blockDim.x) S.W1[k] = P[P_W1 + k];
    for (int k = threadIdx.x; k < BP_H * BP_H; k += blockDim.x) {
        float v = P[P_W2 + k];
        S.W2[k] = v;
        int h = k / BP_H, c = k % BP_H;
        S.W2T[c * BP_H + h] = v;
    }
    for (int k = threadIdx.x; k < BP_H; k += blockDim.x) {
        S.b1[k] = P[P_B1 + k];
        S.b2[k] = P[P_B2 + k];
        S.w3[k] = P[P_W3 + k];
    }
    for (int k = threadIdx.x; k < BP_D; k += blockDim.x) {
        S.mu[k] = norm[k];
        S.sd[k] = norm[BP_D + k];
    }
    if (threadIdx.x == 0) S.b3 = P[P_B3];
    __syncthreads();
}

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// a = M y for a 64x64 matrix held transposed (MT[c][h] = M[h][c]); y is
// distributed as y0 (unit lane) and y1 (unit lane+32); returns the lane's
// two outputs.
__device__ __forceinline__ void matvec64(const float *MT, float y0, float y1, float &o0, float &o1)
{
    const int lane = threadIdx.x & 31;
    o0 = 0.0f;
    o1 = 0.0f;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
        float ya = __shfl_sync(0xffffffffu, y0, c);
        float yb = __shfl_sync(0xffffffffu, y1, c);
        o0 += MT[c * BP_H + lane] * ya + MT[(c + 32) * BP_H + lane] * yb;
        o1 += MT[c * BP_H + lane + 32] * ya + MT[(c + 32) * BP_H + lane + 32] * yb;
    }
}

// x-space input of one atom (all lanes hold all 16 values)
__device__ __forceinline__ void load_x(const MlpSmem &S, const float *G, float x[16])
{
    const float4 *g = reinterpret_cast<const float4 *>(G);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 v = __ldg(g + k);
        x[4 * k] = (v.x - S.mu[4 * k]) / S.sd[4 * k];
        x[4 * k + 1] = (v.y - S.mu[4 * k + 1]) / S.sd[4 * k + 1];
        x[4 * k + 2] = (v.z - S.mu[4 * k + 2]) / S.sd[4 * k + 2];
        x[4 * k + 3] = (v.w - S.mu[4 * k + 3]) / S.sd[4 * k + 3];
    }
}

__device__ __forceinline__ float layer1(const MlpSmem &S, int h, const float x[16])
{
    float a = S.b1[h];
#pragma unroll
    for (int q = 0; q < 16; ++q) a += S.W1[h * BP_D + q] * x[q];
    return a;
}

constexpr int MLP_WARPS = 8;

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_infer(const float *P, const float *norm, const float *G, int N,
                                                             float *Ei, float *dEdG)
{
    count_launch();
    extern __shared__ float4 smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    stage_params(S, P, norm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * MLP_WARPS + w; i < N; i += gridDim.x * MLP_WARPS) {
        float x[16];
        load_x(S, G + (size_t)i * BP_D, x);
        const int h0 = lane, h1 = lane + 32;
        Silu3 s10 = silu3(layer1(S, h0, x)), s11 = silu3(layer1(S, h1, x));
        float a20, a21;
        matvec64(S.W2T, s10.v, s11.v, a20, a21);   // W2 h1
        Silu3 s20 = silu3(a20 + S.b2[h0]), s21 = silu3(a21 + S.b2[h1]);
        float E = wsum(S.w3[h0] * s20.v + S.w3[h1] * s21.v) + S.b3;
        // backward to the input
        float g20 = S.w3[h0] * s20.d1, g21 = S.w3[h1] * s21.d1;
        float t0, t1;
        matvec64(S.W2, g20, g21, t0, t1);           // W2^T g2
        float g10 = t0 * s10.d1, g11 = t1 * s11.d1;
        float dx[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) dx[q] = wsum(S.W1[h0 * BP_D + q] * g10 + S.W1[h1 * BP_D + q] * g11);
        if (lane == 0) {
            Ei[i] = E;
            float4 *o = reinterpret_cast<float4 *>(dEdG + (size_t)i * BP_D);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                o[k] = make_float4(dx[4 * k] / S.sd[4 * k], dx[4 * k + 1] / S.sd[4 * k + 1],
                                   dx[4 * k + 2] / S.sd[4 * k + 2], dx[4 * k + 3] / S.sd[4 * k + 3]);
        }
    }
}

// Per-atom training factors (row a of each):
//   A2 = [d2 | d2t] (128), B2 = [h1 | h1t] (128), A1 = [d1 | d1t] (128),
//   B1 = [x | vt] (32), C3 = c_E h2 - c_F h2t (64)
// so that dW2 = sum A2[:, :64]^T B2[:, :64] + A2[:, 64:]^T B2[:, 64:], etc.
struct TrainOut {
    float *A2, *B2, *A1, *B1, *C3;
};

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_train(const float *P, const float *norm, const float *G,
                                                             const float *V, const float *cE, float cF, int N,
                                                             TrainOut o)
{
    count_launch();
    extern __shared__ float4 smem_raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
    stage_params(S, P, norm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * MLP_WARPS + w; i < N; i += gridDim.x * MLP_WARPS) {
        float x[16], vt[16];
        load_x(S, G + (size_t)i * BP_D, x);
        {
            const float4 *g = reinterpret_cast<const float4 *>(V + (size_t)i * BP_D);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v = __ldg(g + k);
                vt[4 * k] = v.x / S.sd[4 * k];
                vt[4 * k + 1] = v.y / S.sd[4 * k + 1];
                vt[4 * k + 2] = v.z / S.sd[4 * k + 2];
                vt[4 * k + 3] = v.w / S.sd[4 * k + 3];
            }
        }
        const float ce = cE[i];
        const int h0 = lane, h1 = lane + 32;
        // forward and tangent
        Silu3 s10 = silu3(layer1(S, h0, x)), s11 = silu3(layer1(S, h1, x));
        float ad10 = 0.f, ad11 = 0.f;   // W1 vt
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            ad10 += S.W1[h0 * BP_D + q] * vt[q];
            ad11 += S.W1[h1 * BP_D + q] * vt[q];
        }
        float hd10 = s10.d1 * ad10, hd11 = s11.d1 * ad11;
        float a20, a21, ad20, ad21;
        matvec64(S.W2T, s10.v, s11.v, a20, a21);
        matvec64(S.W2T, hd10, hd11, ad20, ad21);
        Silu3 s20 = silu3(a20 + S.b2[h0]), s21 = silu3(a21 + S.b2[h1]);
        float hd20 = s20.d1 * ad20, hd21 = s21.d1 * ad21;
        // reverse through primal and tangent
        const float w30 = S.w3[h0], w31 = S.w3[h1];
        float dd20 = -cF * w30 * s20.d1, dd21 = -cF * w31 * s21.d1;                 // d J / d a2dot
        float d20 = ce * w30 * s20.d1 - cF * w30 * s20.d2 * ad20;                  // d J / d a2
        float d21 = ce * w31 * s21.d1 - cF * w31 * s21.d2 * ad21;
        float u0, u1, ud0, ud1;
        matvec64(S.W2, d20, d21, u0, u1);     // W2^T d2
        matvec64(S.W2, dd20, dd21, ud0, ud1); // W2^T d2dot
        float dd10 = ud0 * s10.d1, dd11 = ud1 * s11.d1;
        float d10 = u0 * s10.d1 + ud0 * s10.d2 * ad10;
        float d11 = u1 * s11.d1 + ud1 * s11.d2 * ad11;
        float *A2 = o.A2 + (size_t)i * 128, *B2 = o.B2 + (size_t)i * 128, *A1 = o.A1 + (size_t)i * 128;
        A2[h0] = d20;
        A2[h1] = d21;
        A2[64 + h0] = dd20;
        A2[64 + h1] = dd21;
        B2[h0] = s10.v;
        B2[h1] = s11.v;
        B2[64 + h0] = hd10;
        B2[64 + h1] = hd11;
        A1[h0] = d10;
        A1[h1] = d11;
        A1[64 + h0] = dd10;
        A1[64 + h1] = dd11;
        float *C3 = o.C3 + (size_t)i * 64;
        C3[h0] = ce * s20.v - cF * hd20;
        C3[h1] = ce * s21.v - cF * hd21;
        if (lane < 16) {
            float xv = 0.f, vv = 0.f;
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (q == lane) {
                    xv = x[q];
                    vv = vt[q];
                }
            o.B1[(size_t)i * 32 + lane] = xv;
            o.B1[(size_t)i * 32 + 16 + lane] = vv;
        }
    }
}

// Weight gradients, one output per thread, atoms summed in order (FP64):
//   dW2[h][c] = sum_a A2[a][h] B2[a][c] + A2[a][64+h] B2[a][64+c]
//   dW1[h][q] = sum_a A1[a][h] B1[a][q] + A1[a][64+h] B1[a][16+q]
//   db2 = sum A2[:, :64], db1 = sum A1[:, :64], dw3 = sum C3, db3 = sum c_E
__global__ void __launch_bounds__(256) k_mlp_grads(TrainOut o, const float *cE, int N, float *grad)
{
    count_launch();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (t < BP_H * BP_H) {
        int h = t / BP_H, c = t % BP_H;
        for (int a = 0; a < N; ++a)
            s += (double)o.A2[(size_t)a * 128 + h] * o.B2[(size_t)a * 128 + c] +
                 (double)o.A2[(size_t)a * 128 + 64 + h] * o.B2[(size_t)a * 128 + 64 + c];
        grad[P_W2 + t] = (float)s;
        return;
    }
    t -= BP_H * BP_H;
    if (t < BP_H * BP_D) {
        int h = t / BP_D, q = t % BP_D;
        for (int a = 0; a < N; ++a)
            s += (double)o.A1[(size_t)a * 128 + h] * o.B1[(size_t)a * 32 + q] +
                 (double)o.A1[(size_t)a * 128 + 64 + h] * o.B1[(size_t)a * 32 + 16 + q];
        grad[P_W1 + t] = (float)s;
        return;
    }
    t -= BP_H * BP_D;
    if (t < BP_H) {
        for (int a = 0; a < N; ++a) s += o.A2[(size_t)a * 128 + t];
        grad[P_B2 + t] = (float)s;
        return;
    }
    t -= BP_H;
    if (t < BP_H) {
        for (int a = 0; a < N; ++a) s += o.A1[(size_t)a * 128 + t];
        grad[P_B1 + t] = (float)s;
        return;
    }
    t -= BP_H;
    if (t < BP_H) {
        for (int a = 0; a < N; ++a) s += o.C3[(size_t)a * 64 + t];
        grad[P_W3 + t] = (float)s;
        return;
    }
    t -= BP_H;
    if (t == 0) {
        for (int a = 0; a < N; ++a) s += cE[a];
        grad[P_B3] = (float)s;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    count_launch();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float gk = g[k];
    float mk = b1 * m[k] + (1.0f - b1) * gk;
    float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Loss bookkeeping for S snapshots of n atoms each (block per snapshot):
//   E_s = sum_i E_i (FP64);  c_E,i = 2 (E_s - E_ref,s) / (S n^2)
//   dF_i = cF (F_i - F_ref,i) with cF = 2 w_F / (3 n S)
//   loss += ((E_s - E_ref,s)/n)^2 / S + w_F |F - F_ref|^2 / (3 n S)
__global__ void __launch_bounds__(256) k_bp_loss_prep(const float *Ei, const float4 *F, const float4 *Fref,
                                                      const double *Eref, int S, int n, float wF, float *cE,
                                                      float4 *dF, double *loss)
{
    count_launch();
    __shared__ double sh[32];
    const int s = blockIdx.x;
    const int b = s * n;
    double e = 0.0, f2 = 0.0;
    const float cF = 2.0f * wF / (3.0f * (float)n * (float)S);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        e += (double)Ei[b + k];
        float4 a = F[b + k], r = Fref[b + k];
        float dx = a.x - r.x, dy = a.y - r.y, dz = a.z - r.z;
        f2 += (double)(dx * dx + dy * dy + dz * dz);
        dF[b + k] = make_float4(cF * dx, cF * dy, cF * dz, 0.0f);
    }
    __shared__ double tot;
    double es = block_sum_f64(e, sh);
    if (threadIdx.x == 0) tot = es;
    __syncthreads();
    const double de = tot - Eref[s];
    const float c = (float)(2.0 * de / ((double)S * (double)n * (double)n));
    for (int k = threadIdx.x; k < n; k += blockDim.x) cE[b + k] = c;
    double fs = block_sum_f64(f2, sh);
    if (threadIdx.x == 0) {
        // per-snapshot terms; the caller sums loss[2 s], loss[2 s + 1]
        loss[2 * s] = de * de / ((double)n * n * S);
        loss[2 * s + 1] = (double)wF * fs / (3.0 * n * S);
    }
}

// Column mean and standard deviation of X [N][D] (FP64, fixed order): one
// block per column.
__global__ void __launch_bounds__(256) k_column_stats(const float *X, int N, int D, float *out)
{
    count_launch();
    __shared__ double sh[32];
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double v = X[(size_t)k * D + c];
        s += v;
        s2 += v * v;
    }
    s = block_sum_f64(s, sh);
    __shared__ double mean;
    if (threadIdx.x == 0) mean = s / N;
    __syncthreads();
    s2 = block_sum_f64(s2, sh);
    if (threadIdx.x == 0) {
        double var = s2 / N - mean * mean;
        out[c] = (float)mean;
        out[D + c] = (float)sqrt(var > 0.0 ? var : 0.0);
    }
}

static int mlp_grid(int N)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
        cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    }
    int groups = (N + MLP_WARPS - 1) / MLP_WARPS;
    int g = sms * 4;
    return groups < g ? groups : g;
}

void enqueue_mlp_infer(const float *P, const float *norm, const float *G, int N, float *Ei, float *dEdG,
                       cudaStream_t st)
{
    int g = mlp_grid(N);
    k_mlp_infer<<<g, MLP_WARPS * 32, sizeof(MlpSmem), st>>>(P, norm, G, N, Ei, dEdG);
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_bp_train_scratch_size(int N)
{
    if (N < 1) return 0;
    const size_t fp32 = (size_t)N * (128 * 3 + 32 + 64) * sizeof(float);   // per-atom factors
    const size_t tc = mlp_train_tc_scratch(N);                               // per-CTA partial gradients
    return fp32 > tc ? fp32 : tc;
}

extern "C" md_status md_bp_mlp_infer(const float *d_params, const float *d_norm, const float *d_G, int N,
                                     float *d_Ei, float *d_dEdG, md_stream_t stream)
{
    if (!d_params || !d_norm || !d_G || !d_Ei || !d_dEdG || N < 1) return MD_ERR_INVALID;
    enqueue_mlp_infer(d_params, d_norm, d_G, N, d_Ei, d_dEdG, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_bp_mlp_train(const float *d_params, const float *d_norm, const float *d_G, const float *d_V,
                                     const float *d_cE, float cF, int N, void *d_scratch, float *d_grad,
                                     md_stream_t stream)
{
    if (!d_params || !d_norm || !d_G || !d_V || !d_cE || !d_scratch || !d_grad || N < 1) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    float *s = (float *)d_scratch;
    TrainOut o;
    o.A2 = s;
    o.B2 = o.A2 + (size_t)N * 128;
    o.A1 = o.B2 + (size_t)N * 128;
    o.B1 = o.A1 + (size_t)N * 128;
    o.C3 = o.B1 + (size_t)N * 32;
    int g = mlp_grid(N);
    k_mlp_train<<<g, MLP_WARPS * 32, sizeof(MlpSmem), st>>>(d_params, d_norm, d_G, d_V, d_cE, cF, N, o);
    int nout = BP_H * BP_H + BP_H * BP_D + 3 * BP_H + 1;
    k_mlp_grads<<<(nout + 255) / 256, 256, 0, st>>>(o, d_cE, N, d_grad);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_bp_loss_prep(const float *d_Ei, const float *d_F, const float *d_Fref, const double *d_Eref,
                                     int S, int n, float wF, float *d_cE, float *d_dF, double *d_loss,
                                     md_stream_t stream)
{
    if (!d_Ei || !d_F || !d_Fref || !d_Eref || !d_cE || !d_dF || !d_loss || S < 1 || n < 1) return MD_ERR_INVALID;
    k_bp_loss_prep<<<S, 256, 0, (cudaStream_t)stream>>>(d_Ei, (const float4 *)d_F, (const float4 *)d_Fref, d_Eref, S,
                                                        n, wF, d_cE, (float4 *)d_dF, d_loss);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_column_stats(const float *d_X, int N, int D, float *d_out, md_stream_t stream)
{
    if (!d_X || !d_out || N < 1 || D < 1) return MD_ERR_INVALID;
    k_column_stats<<<D, 256, 0, (cudaStream_t)stream>>>(d_X, N, D, d_out);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, int n, float lr,
                                  float beta1, float beta2, float eps, int step, md_stream_t stream)
{
    if (!d_params || !d_grad || !d_m || !d_v || n < 1 || step < 1) return MD_ERR_INVALID;
    float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, n, lr, beta1, beta2, eps,
                                                               c1, c2);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
