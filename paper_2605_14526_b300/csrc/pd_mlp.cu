// Learned warm start: training of the 7 -> 128 -> 128 -> 128 -> 3 ReLU
// network (forward, backpropagation, Adam on an FP32 master copy whose
// weights are rounded to BF16 for every forward pass), the per-vertex sample
// kernel (features and targets from a trajectory), the warm-start evaluation
// used by the rollout, and attaching a trained network to a context.
//
// The training GEMMs run on the tensor pipe (mma.sync in TF32 with 3xTF32
// operand splitting, FP32-level accuracy); the elementwise parts on CUDA
// cores. A minibatch of B samples costs about 3 x 35k x B multiply-adds.
// Every reduction has a fixed order, so a training step is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pd_ctx.h"
#include "pd_mlp.cuh"

using namespace pdh;

namespace {

constexpr int H = pdk::kMlpH;
constexpr int NI = pdk::kMlpIn;
constexpr int NO = pdk::kMlpOut;
// flat parameter layout (FP32): W1 [H][7], b1, W2 [H][H], b2, W3 [H][H], b3, W4 [3][H], b4
constexpr int OW1 = 0, OB1 = OW1 + H * NI, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + NO * H, NP = OB4 + NO;
constexpr int NNORM = 2 * NI + NO;

__host__ __device__ inline bool is_weight(int i) {
  return (i >= OW1 && i < OB1) || (i >= OW2 && i < OB2) || (i >= OW3 && i < OB3) || (i >= OW4 && i < OB4);
}

// round-to-nearest-even FP32 -> BF16 bit pattern (finite inputs)
__host__ __device__ inline uint16_t bf16_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__host__ __device__ inline float bf16_value(float x) {
  uint32_t u = (uint32_t)bf16_bits(x) << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// ------------------------------------------------------------ kernels

// C[M][N] (+)= sum_k A(m, k) B(k, n); A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n]. On the tensor pipe: 64 x 64
// tiles, 16-deep slabs staged in shared memory, 8 warps of 16 x 32 outputs,
// mma.sync m16n8k8 in TF32 with each operand split into a TF32 value and its
// TF32 remainder (big + small); the three products big x big, big x small and
// small x big keep FP32-level accuracy ("3xTF32"). Fixed summation order.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32_1688(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Split K: block z of the grid's third dimension takes k in [z kchunk,
// (z + 1) kchunk) and, with part given, writes its partial product to
// part[z][M][N] (summed afterwards in z order by k_splitk_sum).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              int accumulate, int kchunk, float* __restrict__ part) {
  __shared__ float As[16][64 + 8];   // rows of 72: the fragment reads hit 32 distinct banks
  __shared__ float Bs[16][64 + 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = 16 * (warp >> 1), wn = 32 * (warp & 1);   // the warp's 16 x 32 outputs in the tile
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      const int mm = i / 16, kk = i % 16;   // A tile element (m0 + mm, k0 + kk)
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < kend) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
      const int nn = i / 16, kb = i % 16;   // B tile element (k0 + kb, n0 + nn)
      const int n = n0 + nn, kq = k0 + kb;
      Bs[kb][nn] = (n < N && kq < kend) ? (TB ? B[(size_t)n * ldb + kq] : B[(size_t)kq * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k8 = 0; k8 < 16; k8 += 8) {
      const float av[4] = {As[k8 + t][wm + g], As[k8 + t][wm + g + 8], As[k8 + t + 4][wm + g],
                           As[k8 + t + 4][wm + g + 8]};
      uint32_t abig[4], asmall[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        abig[i] = tf32_rna(av[i]);
        asmall[i] = tf32_rna(av[i] - __uint_as_float(abig[i]));
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float b0v = Bs[k8 + t][wn + 8 * j + g], b1v = Bs[k8 + t + 4][wn + 8 * j + g];
        const uint32_t b0 = tf32_rna(b0v), b1 = tf32_rna(b1v);
        const uint32_t s0 = tf32_rna(b0v - __uint_as_float(b0)), s1 = tf32_rna(b1v - __uint_as_float(b1));
        mma_tf32_1688(acc[j], asmall, b0, b1);
        mma_tf32_1688(acc[j], abig, s0, s1);
        mma_tf32_1688(acc[j], abig, b0, b1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + wm + g + (i >= 2 ? 8 : 0), n = n0 + wn + 8 * j + 2 * t + (i & 1);
      if (m < M && n < N) {
        if (part) {
          part[((size_t)blockIdx.z * M + m) * N + n] = acc[j][i];
        } else {
          float* c = C + (size_t)m * ldc + n;
          *c = accumulate ? *c + acc[j][i] : acc[j][i];
        }
      }
    }
}

// C (+)= sum over z of part[z] (fixed order)
__global__ void k_splitk_sum(int M, int N, int splits, const float* __restrict__ part, float* C, int ldc,
                             int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  float v = 0.f;
  for (int z = 0; z < splits; ++z) v += part[(size_t)z * M * N + i];
  float* c = C + (size_t)(i / N) * ldc + i % N;
  *c = accumulate ? *c + v : v;
}

__global__ void k_bias_act(float* Z, const float* b, int n, int N, int relu) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * N) return;
  const float z = Z[i] + b[i % N];
  Z[i] = relu ? fmaxf(z, 0.f) : z;
}

__global__ void k_relu_mask(float* dA, const float* A, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(A[i] > 0.f)) dA[i] = 0.f;
}

// normalised inputs (raw - mean) / scale, FP64 arithmetic then FP32
__global__ void k_normalize(const float* raw, float* out, int n, int width, const float* mean_scale_dev) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * width) return;
  const int c = (int)(i % width);
  out[i] = (float)(((double)raw[i] - (double)mean_scale_dev[c]) / (double)mean_scale_dev[width + c]);
}

// per-component scaling of [n][3] rows: out = in * s[c] (or in / s[c])
__global__ void k_scale3(const float* in, float* out, size_t n3, const float* s, int divide) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const float sc = s[i % NO];
  out[i] = divide ? in[i] / sc : in[i] * sc;
}

// dy = 2 (y - t) / (3n) and per-block partial sums of (y - t)^2
__global__ void __launch_bounds__(256) k_loss(const float* y, const float* t, float* dy, int n, double* part) {
  __shared__ double sh[256];
  const size_t tot = (size_t)n * NO;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)tot;
    s += (double)d * (double)d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// column sums of dZ [n][N] into g[N] (one block per column, fixed order)
__global__ void __launch_bounds__(256) k_colsum(const float* dZ, int n, int N, float* g) {
  __shared__ float sh[256];
  const int j = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s += dZ[(size_t)r * N + j];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) g[j] = sh[0];
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 master copy; the working
// copy gets the weights rounded to BF16 (biases exact)
__global__ void k_adam(float* theta, float* thq, float* m, float* v, const float* g, int n, float lr, float b1,
                       float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  theta[i] = th;
  thq[i] = is_weight(i) ? bf16_value(th) : th;
}

__global__ void k_quantize(const float* theta, float* thq, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) thq[i] = is_weight(i) ? bf16_value(theta[i]) : theta[i];
}

// raw features [x_t - x_{t-1}, x_t - X, log10(E_v / 1e5)] and, if x_{t+1} is
// given, raw targets x_{t+1} - (2 x_t - x_{t-1}), for every vertex
__global__ void k_sample(pdk::Dev d, const double* xtm1, const double* xt, const double* xtp1, float* feat, float* targ) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_v) return;
  for (int i = 0; i < 3; ++i) {
    const size_t o = 3 * (size_t)v + i;
    feat[NI * (size_t)v + i] = (float)(xt[o] - xtm1[o]);
    feat[NI * (size_t)v + 3 + i] = (float)(xt[o] - d.X[o]);
    if (targ && xtp1) targ[NO * (size_t)v + i] = (float)(xtp1[o] - (2.0 * xt[o] - xtm1[o]));
  }
  feat[NI * (size_t)v + 6] = d.logE[v];
}

// q0 of the warm start for every vertex (the network on the tensor pipe, 16
// vertices per warp); pinned vertices at X
__global__ void k_warm_eval(pdk::Dev d, const double* xt, const double* xtm1, double* q0) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v0 = 16 * warp; v0 < d.n_v; v0 += 16 * nwarps) {
    const int v = v0 + (lane & 15);
    if (lane < 16 && v < d.n_v && d.pinned[v])
      for (int i = 0; i < 3; ++i) q0[3 * (size_t)v + i] = d.X[3 * (size_t)v + i];
    pdk::warm_tile(d, v0, xt, xtm1, nullptr, q0, nullptr, lane);
  }
}

inline unsigned blocks(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

constexpr int kSplitMax = 296;   // largest K split (partials of at most 128 x 128 each)

// small M x N with a long K (the weight gradients: K = samples) is split
// over K so that the grid fills the GPU; ws holds kSplitMax x M x N floats
template <bool TA, bool TB>
void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
          int acc = 0, float* ws = nullptr) {
  const int tiles = ((N + 63) / 64) * ((M + 63) / 64);
  int splits = ws && M * N <= 128 * 128 ? std::min(kSplitMax / std::max(tiles, 1), (K + 511) / 512) : 1;
  if (splits < 2) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, 1);
    k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, acc, K, nullptr);
    return;
  }
  const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, 0, kchunk, ws);
  k_splitk_sum<<<(M * N + 255) / 256, 256, 0, s>>>(M, N, splits, ws, C, ldc, acc);
}

}  // namespace

struct pd_mlp {
  int device = 0;
  float* theta = nullptr;   // [NP] FP32 master
  float* thq = nullptr;     // [NP] weights rounded to BF16
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  float* grad = nullptr;    // [NP]
  float* norm_d = nullptr;  // [NNORM]: feature mean, feature scale, output scale
  float norm[NNORM];
  int adam_t = 0;
  float* ws = nullptr;      // per-sample workspace
  size_t ws_rows = 0;
  double* part = nullptr;   // loss partials
  float* skws = nullptr;    // split-K partials of the weight gradients
  std::string err;
};

namespace {

int mfail(pd_mlp* m, int code, const char* msg) {
  if (m) m->err = msg;
  return code;
}

#define MCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return mfail(net, PD_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kLossBlocks = 120;
// per-sample floats of the workspace: a0 [7], a1, a2, a3 [H], y [3], t [3], dy [3], dA, dB [H]
constexpr size_t kWsPerRow = NI + 3 * H + 3 * NO + 2 * H;

int ensure_ws(pd_mlp* net, int64_t n) {
  if ((size_t)n <= net->ws_rows) return PD_OK;
  if (net->ws) cudaFree(net->ws);
  net->ws = nullptr;
  net->ws_rows = 0;
  if (cudaMalloc(&net->ws, (size_t)n * kWsPerRow * sizeof(float)) != cudaSuccess)
    return mfail(net, PD_ERR_OOM, "network workspace allocation");
  net->ws_rows = (size_t)n;
  return PD_OK;
}

struct Acts {
  float *a0, *a1, *a2, *a3, *y, *t, *dy, *dA, *dB;
};

Acts acts(pd_mlp* net, int64_t n) {
  float* p = net->ws;
  Acts a;
  a.a0 = p; p += (size_t)n * NI;
  a.a1 = p; p += (size_t)n * H;
  a.a2 = p; p += (size_t)n * H;
  a.a3 = p; p += (size_t)n * H;
  a.y = p; p += (size_t)n * NO;
  a.t = p; p += (size_t)n * NO;
  a.dy = p; p += (size_t)n * NO;
  a.dA = p; p += (size_t)n * H;
  a.dB = p;
  return a;
}

// forward of n normalised samples in a.a0 with the BF16-rounded weights
void forward(pd_mlp* net, const Acts& a, int n, cudaStream_t s) {
  const float* th = net->thq;
  gemm<false, true>(s, n, H, NI, a.a0, NI, th + OW1, NI, a.a1, H);
  k_bias_act<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.a1, th + OB1, n, H, 1);
  gemm<false, true>(s, n, H, H, a.a1, H, th + OW2, H, a.a2, H);
  k_bias_act<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.a2, th + OB2, n, H, 1);
  gemm<false, true>(s, n, H, H, a.a2, H, th + OW3, H, a.a3, H);
  k_bias_act<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.a3, th + OB3, n, H, 1);
  gemm<false, true>(s, n, NO, H, a.a3, H, th + OW4, H, a.y, NO);
  k_bias_act<<<blocks((size_t)n * NO, 256), 256, 0, s>>>(a.y, th + OB4, n, NO, 0);
}

// loss and gradient of n samples (features and targets raw)
int loss_grad(pd_mlp* net, const float* feat, const float* targ, int n, cudaStream_t s, double* loss) {
  int r;
  if ((r = ensure_ws(net, n))) return r;
  const Acts a = acts(net, n);
  k_normalize<<<blocks((size_t)n * NI, 256), 256, 0, s>>>(feat, a.a0, n, NI, net->norm_d);
  // targets: raw / oscale
  k_scale3<<<blocks((size_t)n * NO, 256), 256, 0, s>>>(targ, a.t, (size_t)n * NO, net->norm_d + 2 * NI, 1);
  forward(net, a, n, s);
  k_loss<<<kLossBlocks, 256, 0, s>>>(a.y, a.t, a.dy, n, net->part);
  const float* th = net->thq;
  float* g = net->grad;
  // output layer
  gemm<true, false>(s, NO, H, n, a.dy, NO, a.a3, H, g + OW4, H, 0, net->skws);
  k_colsum<<<NO, 256, 0, s>>>(a.dy, n, NO, g + OB4);
  gemm<false, false>(s, n, H, NO, a.dy, NO, th + OW4, H, a.dA, H);
  k_relu_mask<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.dA, a.a3, (size_t)n * H);
  // layer 3
  gemm<true, false>(s, H, H, n, a.dA, H, a.a2, H, g + OW3, H, 0, net->skws);
  k_colsum<<<H, 256, 0, s>>>(a.dA, n, H, g + OB3);
  gemm<false, false>(s, n, H, H, a.dA, H, th + OW3, H, a.dB, H);
  k_relu_mask<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.dB, a.a2, (size_t)n * H);
  // layer 2
  gemm<true, false>(s, H, H, n, a.dB, H, a.a1, H, g + OW2, H, 0, net->skws);
  k_colsum<<<H, 256, 0, s>>>(a.dB, n, H, g + OB2);
  gemm<false, false>(s, n, H, H, a.dB, H, th + OW2, H, a.dA, H);
  k_relu_mask<<<blocks((size_t)n * H, 256), 256, 0, s>>>(a.dA, a.a1, (size_t)n * H);
  // layer 1
  gemm<true, false>(s, H, NI, n, a.dA, H, a.a0, NI, g + OW1, NI, 0, net->skws);
  k_colsum<<<H, 256, 0, s>>>(a.dA, n, H, g + OB1);
  if (cudaGetLastError() != cudaSuccess) return mfail(net, PD_ERR_CUDA, "network kernel launch failed");
  if (loss) {
    double hp[kLossBlocks];
    MCK(cudaMemcpyAsync(hp, net->part, sizeof(hp), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    double L = 0.0;
    for (int i = 0; i < kLossBlocks; ++i) L += hp[i];
    *loss = L / ((double)n * NO);
  }
  return PD_OK;
}

}  // namespace

extern "C" {

int pd_mlp_create(const float* theta, const float* norm, pd_mlp** out) {
  if (!out || !theta || !norm) return PD_ERR_ARG;
  *out = nullptr;
  pd_mlp* net = new pd_mlp();
  *out = net;
  MCK(cudaGetDevice(&net->device));
  for (int i = 0; i < NNORM; ++i) {
    net->norm[i] = norm[i];
    if (!std::isfinite(norm[i]) || (i >= NI && !(norm[i] > 0))) return mfail(net, PD_ERR_ARG, "invalid normalisation");
  }
  float** bufs[] = {&net->theta, &net->thq, &net->m, &net->v, &net->grad};
  for (float** b : bufs) {
    MCK(cudaMalloc(b, NP * sizeof(float)));
    MCK(cudaMemset(*b, 0, NP * sizeof(float)));
  }
  MCK(cudaMalloc(&net->norm_d, NNORM * sizeof(float)));
  MCK(cudaMalloc(&net->part, kLossBlocks * sizeof(double)));
  MCK(cudaMalloc(&net->skws, (size_t)kSplitMax * H * H * sizeof(float)));
  MCK(cudaMemcpy(net->theta, theta, NP * sizeof(float), cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(net->norm_d, net->norm, NNORM * sizeof(float), cudaMemcpyHostToDevice));
  k_quantize<<<blocks(NP, 256), 256>>>(net->theta, net->thq, NP);
  MCK(cudaGetLastError());
  MCK(cudaDeviceSynchronize());
  return PD_OK;
}

int pd_mlp_params(const pd_mlp* net, float* theta, float* norm) {
  if (!net) return PD_ERR_ARG;
  if (theta && cudaMemcpy(theta, net->theta, NP * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PD_ERR_CUDA;
  if (norm) std::memcpy(norm, net->norm, sizeof(net->norm));
  return PD_OK;
}

int pd_mlp_fit_normalization(pd_mlp* net, const float* feat, const float* targ, int64_t n, void* stream) {
  if (!net || !feat || !targ || n < 1) return PD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> hf((size_t)n * NI), ht((size_t)n * NO);
  MCK(cudaMemcpyAsync(hf.data(), feat, hf.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
  MCK(cudaMemcpyAsync(ht.data(), targ, ht.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  for (int c = 0; c < NI; ++c) {
    double mu = 0.0, var = 0.0;
    for (int64_t r = 0; r < n; ++r) mu += hf[(size_t)r * NI + c];
    mu /= (double)n;
    for (int64_t r = 0; r < n; ++r) var += (hf[(size_t)r * NI + c] - mu) * (hf[(size_t)r * NI + c] - mu);
    const double sd = std::sqrt(var / (double)n);
    net->norm[c] = (float)mu;
    net->norm[NI + c] = sd > 1e-12 ? (float)sd : 1.f;
  }
  for (int c = 0; c < NO; ++c) {
    double ms = 0.0;
    for (int64_t r = 0; r < n; ++r) ms += (double)ht[(size_t)r * NO + c] * ht[(size_t)r * NO + c];
    const double rms = std::sqrt(ms / (double)n);
    net->norm[2 * NI + c] = rms > 1e-12 ? (float)rms : 1.f;
  }
  MCK(cudaMemcpyAsync(net->norm_d, net->norm, NNORM * sizeof(float), cudaMemcpyHostToDevice, s));
  MCK(cudaStreamSynchronize(s));
  return PD_OK;
}

int pd_mlp_forward(pd_mlp* net, const float* feat, float* r, int64_t n, void* stream) {
  if (!net || !feat || !r || n < 1 || n > 0x7fffffff) return PD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = ensure_ws(net, n))) return rc;
  const Acts a = acts(net, n);
  k_normalize<<<blocks((size_t)n * NI, 256), 256, 0, s>>>(feat, a.a0, (int)n, NI, net->norm_d);
  forward(net, a, (int)n, s);
  k_scale3<<<blocks((size_t)n * NO, 256), 256, 0, s>>>(a.y, r, (size_t)n * NO, net->norm_d + 2 * NI, 0);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(s));
  return PD_OK;
}

int pd_mlp_grad(pd_mlp* net, const float* feat, const float* targ, int64_t n, float* grad, double* loss, void* stream) {
  if (!net || !feat || !targ || n < 1 || n > 0x7fffffff) return PD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(net, feat, targ, (int)n, s, loss);
  if (rc) return rc;
  if (grad) MCK(cudaMemcpyAsync(grad, net->grad, NP * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MCK(cudaStreamSynchronize(s));
  return PD_OK;
}

int pd_mlp_train_step(pd_mlp* net, const float* feat, const float* targ, int64_t n, double lr, double* loss,
                      void* stream) {
  if (!net || !feat || !targ || n < 1 || n > 0x7fffffff || !(lr > 0)) return PD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(net, feat, targ, (int)n, s, loss);
  if (rc) return rc;
  net->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float bc1 = (float)(1.0 - std::pow(0.9, net->adam_t)), bc2 = (float)(1.0 - std::pow(0.999, net->adam_t));
  k_adam<<<blocks(NP, 256), 256, 0, s>>>(net->theta, net->thq, net->m, net->v, net->grad, NP, (float)lr, b1, b2, eps,
                                         bc1, bc2);
  MCK(cudaGetLastError());
  return PD_OK;
}

const char* pd_mlp_last_error(const pd_mlp* net) { return net ? net->err.c_str() : "null network"; }

void pd_mlp_destroy(pd_mlp* net) {
  if (!net) return;
  float* bufs[] = {net->theta, net->thq, net->m, net->v, net->grad, net->norm_d, net->ws};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (net->part) cudaFree(net->part);
  if (net->skws) cudaFree(net->skws);
  delete net;
}

int pd_mlp_sample(pd_ctx* c, const double* x_tm1, const double* x_t, const double* x_tp1, float* feat, float* targ,
                  void* stream) {
  if (!c || !x_tm1 || !x_t || !feat) return PD_ERR_ARG;
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_mlp_sample");
  CK(cudaSetDevice(c->device));
  if (c->batch) {   // the concatenated arrays of a batch: one launch per instance
    for (int i = 0; i < batch_size(c); ++i) {
      int64_t vo = 0;
      const pd_ctx* k = batch_kid(c, i, &vo);
      k_sample<<<blocks(k->n_v, 256), 256, 0, (cudaStream_t)stream>>>(
          k->d, x_tm1 + 3 * vo, x_t + 3 * vo, x_tp1 ? x_tp1 + 3 * vo : nullptr, feat + (size_t)NI * vo,
          targ ? targ + (size_t)NO * vo : nullptr);
    }
    CK(cudaGetLastError());
    c->launches += batch_size(c);
    return PD_OK;
  }
  k_sample<<<blocks(c->n_v, 256), 256, 0, (cudaStream_t)stream>>>(c->d, x_tm1, x_t, x_tp1, feat, targ);
  CK(cudaGetLastError());
  c->launches += 1;
  return PD_OK;
}

int pd_set_warm_start(pd_ctx* c, int32_t mode) {
  if (!c) return PD_ERR_ARG;
  if (mode < 0 || mode > 2) return fail(c, PD_ERR_ARG, "warm_start must be 0, 1 or 2");
  if (mode != 0 && !c->opt.persistent) return fail(c, PD_ERR_ARG, "the warm start needs persistent launches");
  if (mode == 1 && !(c->batch ? batch_has_mlp(c) : c->d.mlp.w != nullptr))
    return fail(c, PD_ERR_ARG, "warm_start = 1 needs a network (pd_mlp_load)");
  c->opt.warm_start = mode;
  c->d.warm = mode;
  if (c->batch) batch_set_warm(c, mode);
  return PD_OK;
}

int pd_warm_start(pd_ctx* c, const double* x_t, const double* x_tm1, double* q0, void* stream) {
  if (!c || !x_t || !x_tm1 || !q0) return PD_ERR_ARG;
  if (c->batch) return fail(c, PD_ERR_ARG, "pd_warm_start is single-instance only");
  if (!c->factored) return fail(c, PD_ERR_NOT_FACTORED, "pd_factor must run before pd_warm_start");
  if (c->opt.warm_start == 1 && !c->d.mlp.w) return fail(c, PD_ERR_ARG, "no network loaded (pd_mlp_load)");
  CK(cudaSetDevice(c->device));
  pdk::Dev d = c->d;
  d.warm = c->opt.warm_start ? c->opt.warm_start : 1;
  if (d.warm == 1 && !d.mlp.w) return fail(c, PD_ERR_ARG, "no network loaded (pd_mlp_load)");
  k_warm_eval<<<blocks(2 * (size_t)c->n_v + 32, 256), 256, 0, (cudaStream_t)stream>>>(d, x_t, x_tm1, q0);
  CK(cudaGetLastError());
  c->launches += 1;
  return PD_OK;
}

}  // extern "C"

// network blob (FP32 parameters [NP] then normalisation [NNORM]) -> the
// kernels' layout: BF16 weights input-major, FP32 biases
int mlp_upload(pd_ctx* c, const void* blob, size_t bytes, pdk::MlpDev* out, std::vector<void*>& owner) {
  if (bytes != (size_t)(NP + NNORM) * sizeof(float)) return fail(c, PD_ERR_ARG, "network blob must hold %d floats", NP + NNORM);
  const float* th = reinterpret_cast<const float*>(blob);
  const float* nm = th + NP;
  for (int i = 0; i < NP + NNORM; ++i)
    if (!std::isfinite(th[i])) return fail(c, PD_ERR_ARG, "non-finite network parameter %d", i);
  for (int i = NI; i < NNORM; ++i)
    if (!(nm[i] > 0)) return fail(c, PD_ERR_ARG, "normalisation scales must be > 0");
  std::vector<uint16_t> w(pdk::kMlpWeights);
  std::vector<float> b(pdk::kMlpBiases);
  size_t o = 0;
  for (int k = 0; k < NI; ++k)
    for (int j = 0; j < H; ++j) w[o++] = bf16_bits(th[OW1 + j * NI + k]);
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < H; ++j) w[o++] = bf16_bits(th[OW2 + j * H + k]);
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < H; ++j) w[o++] = bf16_bits(th[OW3 + j * H + k]);
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < NO; ++j) w[o++] = bf16_bits(th[OW4 + j * H + k]);
  for (int j = 0; j < H; ++j) {
    b[j] = th[OB1 + j];
    b[H + j] = th[OB2 + j];
    b[2 * H + j] = th[OB3 + j];
  }
  for (int j = 0; j < NO; ++j) b[3 * H + j] = th[OB4 + j];
  // the tensor-core copy: B fragments of mma.sync m16n8k16 per layer
  std::vector<uint2> wf(pdk::kMlpFrags);
  {
    size_t f = 0;
    auto pack = [&](int ow, int K, int N, int ksteps, int ntiles) {
      auto wv = [&](int k, int n) -> uint32_t { return (k < K && n < N) ? bf16_bits(th[ow + n * K + k]) : 0u; };
      for (int ks = 0; ks < ksteps; ++ks)
        for (int nt = 0; nt < ntiles; ++nt)
          for (int lane = 0; lane < 32; ++lane) {
            const int t = lane & 3, n = 8 * nt + (lane >> 2), k = 16 * ks + 2 * t;
            wf[f++] = make_uint2(wv(k, n) | wv(k + 1, n) << 16, wv(k + 8, n) | wv(k + 9, n) << 16);
          }
    };
    pack(OW1, NI, H, 1, 16);
    pack(OW2, H, H, 8, 16);
    pack(OW3, H, H, 8, 16);
    pack(OW4, H, NO, 8, 1);
  }
  uint16_t* wd = nullptr;
  uint2* wfd = nullptr;
  float* bd = nullptr;
  CK(cudaMalloc(&wd, w.size() * sizeof(uint16_t)));
  owner.push_back(wd);
  CK(cudaMalloc(&wfd, wf.size() * sizeof(uint2)));
  owner.push_back(wfd);
  CK(cudaMemcpy(wfd, wf.data(), wf.size() * sizeof(uint2), cudaMemcpyHostToDevice));
  out->wf = wfd;
  CK(cudaMalloc(&bd, b.size() * sizeof(float)));
  owner.push_back(bd);
  CK(cudaMemcpy(wd, w.data(), w.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(bd, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice));
  out->w = wd;
  out->b = bd;
  for (int i = 0; i < NI; ++i) {
    out->fmean[i] = nm[i];
    out->fscale[i] = nm[NI + i];
  }
  for (int i = 0; i < NO; ++i) out->oscale[i] = nm[2 * NI + i];
  return PD_OK;
}
