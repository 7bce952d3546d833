// Training, packing, guard and stand-alone evaluation kernels of the learned Voigt
// surrogate (not part of the paper; the network and its contract are described in
// mlp.cuh).
//
// Training runs in FP32 on the CUDA cores: a block takes kTrainTile samples with one
// thread per hidden unit, keeps the tile's activations in shared memory, and writes its
// partial weight gradient; the partials are summed over blocks in a fixed order
// (deterministic), then Adam updates the parameters. With qat set, the forward pass
// rounds W2, W3 and the layer-1 and layer-2 activations to BF16 as the tensor-core
// inference does, and the backward pass treats the rounding as the identity (the
// straight-through estimator), so the network is trained for the precision it runs in.
#include "mlp.cuh"

namespace marfa {

constexpr int kH = kMlpH;
constexpr int kTrainTile = 16;
int mlp_train_tile() { return kTrainTile; }

__device__ __forceinline__ float silu_ref(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_ref(float z) {
  const float sg = 1.0f / (1.0f + expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}
__device__ __forceinline__ float bf_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__global__ void __launch_bounds__(kH)
    k_mlp_fwd_bwd(const float* __restrict__ W, const float* __restrict__ xs, const float* __restrict__ ys,
                  const float* __restrict__ ts, int64_t n, int64_t first, float inv_batch, int qat,
                  float* __restrict__ part, float* __restrict__ loss_part) {
  constexpr int S = kTrainTile;
  __shared__ float U[S][2];
  __shared__ float Z1[S][kH], A1[S][kH], Z2[S][kH], A2[S][kH], Z3[S][kH], A3[S][kH];
  __shared__ float D4[S];
  __shared__ float D[S][kH];  // dL/dz of the current layer, per sample
  const int h = threadIdx.x;
  const int64_t s0 = first + (int64_t)blockIdx.x * S;
  if (h < S) {
    const int64_t i = s0 + h;
    float u1 = 0.f, u2 = 0.f;
    if (i < n) {
      u1 = logf(ys[i]);
      u2 = log1pf(fabsf(xs[i]) / (1.0f + ys[i]));
    }
    U[h][0] = u1;
    U[h][1] = u2;
  }
  __syncthreads();
  // forward: thread h computes hidden unit h of every sample of the tile
  {
    const float w0 = W[kMlpOffW1 + 2 * h], w1 = W[kMlpOffW1 + 2 * h + 1], b = W[kMlpOffB1 + h];
    for (int s = 0; s < S; ++s) {
      const float z = fmaf(w0, U[s][0], fmaf(w1, U[s][1], b));
      Z1[s][h] = z;
      A1[s][h] = qat ? bf_round(silu_ref(z)) : silu_ref(z);
    }
  }
  __syncthreads();
  {
    float z[S];
    const float b = W[kMlpOffB2 + h];
    for (int s = 0; s < S; ++s) z[s] = b;
    for (int k = 0; k < kH; ++k) {
      const float w = qat ? bf_round(W[kMlpOffW2 + h * kH + k]) : W[kMlpOffW2 + h * kH + k];
      for (int s = 0; s < S; ++s) z[s] = fmaf(w, A1[s][k], z[s]);
    }
    for (int s = 0; s < S; ++s) {
      Z2[s][h] = z[s];
      A2[s][h] = qat ? bf_round(silu_ref(z[s])) : silu_ref(z[s]);
    }
  }
  __syncthreads();
  {
    float z[S];
    const float b = W[kMlpOffB3 + h];
    for (int s = 0; s < S; ++s) z[s] = b;
    for (int k = 0; k < kH; ++k) {
      const float w = qat ? bf_round(W[kMlpOffW3 + h * kH + k]) : W[kMlpOffW3 + h * kH + k];
      for (int s = 0; s < S; ++s) z[s] = fmaf(w, A2[s][k], z[s]);
    }
    for (int s = 0; s < S; ++s) {
      Z3[s][h] = z[s];
      A3[s][h] = silu_ref(z[s]);
    }
  }
  __syncthreads();
  if (h < S) {
    const int64_t i = s0 + h;
    float t = W[kMlpOffB4];
    for (int k = 0; k < kH; ++k) t = fmaf(W[kMlpOffW4 + k], A3[h][k], t);
    const float r = i < n ? t - ts[i] : 0.0f;
    D4[h] = 2.0f * r * inv_batch;  // dL/dt with L = mean of r^2 over the batch
    loss_part[(int64_t)blockIdx.x * S + h] = r * r;
  }
  __syncthreads();
  float* g = part + (int64_t)blockIdx.x * kMlpParams;
  // output layer
  {
    float gw = 0.f, gb = 0.f;
    const float w4 = W[kMlpOffW4 + h];
    for (int s = 0; s < S; ++s) {
      gw = fmaf(D4[s], A3[s][h], gw);
      gb += D4[s];
      D[s][h] = D4[s] * w4 * dsilu_ref(Z3[s][h]);
    }
    g[kMlpOffW4 + h] = gw;
    if (h == 0) g[kMlpOffB4] = gb;
  }
  __syncthreads();
  // hidden layers 3 and 2: dW[h][k] = sum_s d[s][h] a_in[s][k]; d_in = W^T d * silu'(z_in)
  for (int layer = 3; layer >= 2; --layer) {
    const int offW = layer == 3 ? kMlpOffW3 : kMlpOffW2, offB = layer == 3 ? kMlpOffB3 : kMlpOffB2;
    float (*Ain)[kH] = layer == 3 ? A2 : A1;
    float (*Zin)[kH] = layer == 3 ? Z2 : Z1;
    float gb = 0.f;
    for (int s = 0; s < S; ++s) gb += D[s][h];
    g[offB + h] = gb;
    for (int k = 0; k < kH; ++k) {
      float acc = 0.f;
      for (int s = 0; s < S; ++s) acc = fmaf(D[s][h], Ain[s][k], acc);
      g[offW + h * kH + k] = acc;
    }
    float nd[S];
    for (int s = 0; s < S; ++s) nd[s] = 0.f;
    for (int o = 0; o < kH; ++o) {
      const float w = qat ? bf_round(W[offW + o * kH + h]) : W[offW + o * kH + h];
      for (int s = 0; s < S; ++s) nd[s] = fmaf(w, D[s][o], nd[s]);
    }
    __syncthreads();
    for (int s = 0; s < S; ++s) D[s][h] = nd[s] * dsilu_ref(Zin[s][h]);
    __syncthreads();
  }
  // layer 1
  {
    float gb = 0.f, g0 = 0.f, g1 = 0.f;
    for (int s = 0; s < S; ++s) {
      gb += D[s][h];
      g0 = fmaf(D[s][h], U[s][0], g0);
      g1 = fmaf(D[s][h], U[s][1], g1);
    }
    g[kMlpOffB1 + h] = gb;
    g[kMlpOffW1 + 2 * h] = g0;
    g[kMlpOffW1 + 2 * h + 1] = g1;
  }
}

// grad[j] = compensated sum over blocks of part[b][j], in block order
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kMlpParams) return;
  float s = 0.f, c = 0.f;
  for (int b = 0; b < nblk; ++b) {
    const float v = part[(int64_t)b * kMlpParams + j] - c;
    const float t = s + v;
    c = (t - s) - v;
    s = t;
  }
  grad[j] = s;
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1t, float b2t) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mj = b1 * m[j] + (1.0f - b1) * g[j];
  const float vj = b2 * v[j] + (1.0f - b2) * g[j] * g[j];
  m[j] = mj;
  v[j] = vj;
  p[j] -= lr * (mj / (1.0f - b1t)) / (sqrtf(vj / (1.0f - b2t)) + eps);
}

// out[0] = inv * sum of lp[0 .. n-1] (one block, fixed order)
__global__ void __launch_bounds__(256) k_mlp_loss_sum(const float* __restrict__ lp, int n, float inv,
                                                      float* __restrict__ out) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += 256) s += lp[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * inv;
}

void launch_mlp_loss_sum(const float* lp, int n, float inv, float* out, cudaStream_t st) {
  k_mlp_loss_sum<<<1, 256, 0, st>>>(lp, n, inv, out);
}

void launch_mlp_fwd_bwd(const float* params, const float* x, const float* y, const float* t, int64_t n,
                        int64_t first, int nblk, float inv_batch, bool qat, float* part, float* loss_part,
                        cudaStream_t st) {
  k_mlp_fwd_bwd<<<nblk, kH, 0, st>>>(params, x, y, t, n, first, inv_batch, qat ? 1 : 0, part, loss_part);
}
void launch_mlp_reduce(const float* part, int nblk, float* grad, cudaStream_t st) {
  k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, st>>>(part, nblk, grad);
}
void launch_mlp_adam(float* p, const float* g, float* m, float* v, float lr, float b1t, float b2t,
                     cudaStream_t st) {
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, g, m, v, lr, b1t, b2t);
}

// ------------------------------------------------------------------ inference weights
// FP32 training parameters -> MlpWeights (W2, W3 rounded to BF16, rows padded; guard
// cleared).
__global__ void k_mlp_pack(const float* __restrict__ p, MlpWeights* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * kH) out->w1[j] = p[kMlpOffW1 + j];
  if (j < kH) {
    out->b1[j] = p[kMlpOffB1 + j];
    out->b2[j] = p[kMlpOffB2 + j];
    out->b3[j] = p[kMlpOffB3 + j];
    out->w4[j] = p[kMlpOffW4 + j];
  }
  if (j < 3) out->pad[j] = 0.0f;
  if (j == 0) out->b4 = p[kMlpOffB4];
  if (j < kH * kWStride) {
    const int o = j / kWStride, i = j % kWStride;
    const float w2 = i < kH ? p[kMlpOffW2 + o * kH + i] : 0.0f;
    const float w3 = i < kH ? p[kMlpOffW3 + o * kH + i] : 0.0f;
    out->w2[j] = __bfloat16_as_ushort(__float2bfloat16_rn(w2));
    out->w3[j] = __bfloat16_as_ushort(__float2bfloat16_rn(w3));
  }
  if (j < kGuardWords) out->guard[j] = 0u;
}

void launch_mlp_pack(const float* p, MlpWeights* out, cudaStream_t st) {
  k_mlp_pack<<<(kH * kWStride + 255) / 256, 256, 0, st>>>(p, out);
}

// ------------------------------------------------------------------ guard
// One warp per guard cell. The cell is eligible when it lies inside the training domain
// (1e-4 <= y <= 10) and inside the region where the plain FP32 Voigt takes its costly
// branches (y < 1, or y >= 1 with x^2 + y^2 < 64 at the cell's far corner). The warp
// evaluates the surrogate and the plain Voigt on an n x n lattice spanning the cell,
// edges included, and sets the cell's bit when every lattice point agrees within the
// relative budget. cell_err receives the largest relative difference (-1 if not eligible).
__global__ void __launch_bounds__(128) k_mlp_guard(MlpWeights* __restrict__ w, float budget, int nsamp,
                                                   float* __restrict__ cell_err) {
  __shared__ MlpWeights S;
  mlp_load_smem(S, w);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int cell = blockIdx.x * 4 + (threadIdx.x >> 5);  // warp-uniform
  if (cell >= kGuardNx * kGuardNy) return;
  const int ix = cell % kGuardNx, iy = cell / kGuardNx;
  const int e = iy / 4 - 14, k = iy % 4;
  const float xl = ix * 0.125f, xh = (ix + 1) * 0.125f;
  const float yl = ldexpf(1.0f + 0.25f * k, e), yh = ldexpf(1.0f + 0.25f * (k + 1), e);
  const bool eligible = yl >= 1e-4f && yh <= 10.0f && (yh <= 1.0f || xh * xh + yh * yh < 64.0f);
  float worst = -1.0f;
  if (eligible) {
    worst = 0.0f;
    const int tot = nsamp * nsamp;
    for (int b = 0; b < tot; b += 32) {  // warp-uniform trip count
      const int q = b + lane;
      const bool act = q < tot;
      const int a = act ? q % nsamp : 0, c = act ? q / nsamp : 0;
      // the top edge of each cell is approached to within one part in 2^20
      const float fa = (float)a / (float)(nsamp - 1), fc = (float)c / (float)(nsamp - 1);
      const float x = fminf(fmaf(fa, xh - xl, xl), xh * (1.0f - 0x1p-20f));
      const float y = fminf(fmaf(fc, yh - yl, yl), yh * (1.0f - 0x1p-20f));
      const float ks = mlp_warp_K(S, x, y);
      const float kp = voigt_K(x, y);
      const float r = act ? fabsf(ks / kp - 1.0f) : 0.0f;
      worst = fmaxf(worst, r == r ? r : 1e30f);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  }
  if (lane == 0) {
    if (cell_err) cell_err[cell] = worst;
    if (eligible && worst <= budget) atomicOr(&w->guard[cell >> 5], 1u << (cell & 31));
  }
}

void launch_mlp_guard(MlpWeights* w, float budget, int samples, float* cell_err, cudaStream_t st) {
  const int cells = kGuardNx * kGuardNy;
  k_mlp_guard<<<(cells + 3) / 4, 128, 0, st>>>(w, budget, samples, cell_err);
}

// ------------------------------------------------------------------ evaluation
// out[i] = surrogate K(x[i], y[i]) (guarded = false), or the guarded evaluation the
// profile kernels use: the surrogate where the guard holds, the plain FP32 Voigt elsewhere.
__global__ void __launch_bounds__(128) k_mlp_eval(const MlpWeights* __restrict__ w, const float* __restrict__ x,
                                                  const float* __restrict__ y, float* __restrict__ out,
                                                  int64_t n, int guarded) {
  __shared__ MlpWeights S;
  mlp_load_smem(S, w);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < n;
  const float xi = act ? x[i] : 0.0f, yi = act ? y[i] : 1.0f;
  float k;
  if (guarded) {
    int64_t nm = 0;
    k = voigt_K_coll<false>(xi, yi, act, kVoigtCells, S, nm);
  } else {
    k = mlp_warp_K(S, xi, yi);
  }
  if (act) out[i] = k;
}

void launch_mlp_eval(const MlpWeights* w, const float* x, const float* y, float* out, int64_t n, bool guarded,
                     cudaStream_t st) {
  if (n <= 0) return;
  k_mlp_eval<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(w, x, y, out, n, guarded ? 1 : 0);
}

}  // namespace marfa
