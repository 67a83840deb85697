// Training and evaluation of the learned Fermi-Dirac inversion (the network
// of surrogate.cuh), with the project's own kernels:
//  * targets_kernel: exact forward map of the method, (n, t) -> embedded
//    inputs (n_hat, l_hat) of (n, e) and normalised targets (ln T, mu), FP64,
//    stored FP32;
//  * fwd_bwd_kernel: one sample per thread, activations of a 128-sample
//    block in shared memory, backpropagation, then the block's partial weight
//    gradients (fixed-order sums over its samples);
//  * grad_reduce_kernel: partials summed over blocks in a fixed order;
//  * adam_kernel: Adam update (Kingma and Ba, 2015) with a cosine learning
//    rate schedule.
// Every sum runs in a fixed order, so training is bit-for-bit repeatable.
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "fd_device.cuh"
#include "lbm.h"
#include "surrogate.cuh"

namespace {

using namespace lbm;

constexpr int kBT = 128;   // samples per training block
constexpr int kLd = kH + 1;  // padded row of the activation tiles

// shared layout of fwd_bwd_kernel (floats)
constexpr int kSmW = 0;
constexpr int kSmH1 = kSmW + kNParam;
constexpr int kSmZ2 = kSmH1 + kBT * kLd;
constexpr int kSmDZ2 = kSmZ2 + kBT * kLd;
constexpr int kSmDZ1 = kSmDZ2 + kBT * kLd;
constexpr int kSmX = kSmDZ1 + kBT * kLd;
constexpr int kSmD = kSmX + 2 * kBT;
constexpr int kSmL = kSmD + 2 * kBT;
constexpr int kSmTotal = kSmL + kBT;

__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ float silu_exact(float z) { return z / (1.0f + expf(-z)); }

__global__ void targets_kernel(const double* __restrict__ n, const double* __restrict__ t, int64_t count,
                               float* __restrict__ feat, float* __restrict__ targ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double nn = n[i], tt = t[i];
  const double x = x_of_t(tt);
  const double J2 = j2_of(fd_eval(x));
  const double e = 2.0 * nn * J2 / 3.0;
  const double T = nn * tt / (2.0 * kPi);
  const double mu = T * x;
  const double delta = 1.5 - 1.5 * e / nn;
  feat[2 * i] = (float)((nn - (double)kSurNMid) / (double)kSurNHalf);
  feat[2 * i + 1] = (float)((log(delta) - (double)kSurLdMid) / (double)kSurLdHalf);
  targ[2 * i] = (float)((log(T) - (double)kSurLnTMid) / (double)kSurLnTHalf);
  targ[2 * i + 1] = (float)((mu - (double)kSurMuMid) / (double)kSurMuHalf);
}

// Loss sum_o (y_o - target_o)^2 averaged over `scale_count` samples.
__global__ void __launch_bounds__(kBT) fwd_bwd_kernel(const float* __restrict__ params, const float* __restrict__ feat,
                                                      const float* __restrict__ targ, int64_t begin, int64_t count,
                                                      float inv_batch, float* __restrict__ partials,
                                                      float* __restrict__ loss_partials) {
  extern __shared__ float sm[];
  float* sW = sm + kSmW;
  float* sH1 = sm + kSmH1;
  float* sZ2 = sm + kSmZ2;
  float* sDZ2 = sm + kSmDZ2;
  float* sDZ1 = sm + kSmDZ1;
  float* sX = sm + kSmX;
  float* sD = sm + kSmD;
  float* sL = sm + kSmL;
  const int tid = threadIdx.x;
  for (int e = tid; e < kNParam; e += kBT) sW[e] = params[e];
  const int64_t s = begin + (int64_t)blockIdx.x * kBT + tid;
  const bool valid = s < begin + count;
  const float x0 = valid ? feat[2 * s] : 0.0f, x1 = valid ? feat[2 * s + 1] : 0.0f;
  const float y0 = valid ? targ[2 * s] : 0.0f, y1 = valid ? targ[2 * s + 1] : 0.0f;
  sX[2 * tid] = x0;
  sX[2 * tid + 1] = x1;
  __syncthreads();
  // forward
  for (int k = 0; k < kH; ++k) {
    const float z = sW[kOW1 + 2 * k] * x0 + sW[kOW1 + 2 * k + 1] * x1 + sW[kOB1 + k];
    sH1[tid * kLd + k] = silu_exact(z);
  }
  float o0 = sW[kOB3], o1 = sW[kOB3 + 1];
  for (int j = 0; j < kH; ++j) {
    float z = sW[kOB2 + j];
    for (int k = 0; k < kH; ++k) z += sW[kOW2 + kH * j + k] * sH1[tid * kLd + k];
    sZ2[tid * kLd + j] = z;
    const float h = silu_exact(z);
    o0 += sW[kOW3 + j] * h;
    o1 += sW[kOW3 + kH + j] * h;
  }
  const float r0 = valid ? o0 - y0 : 0.0f, r1 = valid ? o1 - y1 : 0.0f;
  const float d0 = 2.0f * r0 * inv_batch, d1 = 2.0f * r1 * inv_batch;
  sD[2 * tid] = d0;
  sD[2 * tid + 1] = d1;
  sL[tid] = r0 * r0 + r1 * r1;
  // backward
  for (int j = 0; j < kH; ++j) {
    const float dh = sW[kOW3 + j] * d0 + sW[kOW3 + kH + j] * d1;
    sDZ2[tid * kLd + j] = dh * dsilu_f(sZ2[tid * kLd + j]);
  }
  for (int k = 0; k < kH; ++k) {
    float dh = 0.0f;
    for (int j = 0; j < kH; ++j) dh += sW[kOW2 + kH * j + k] * sDZ2[tid * kLd + j];
    const float z1 = sW[kOW1 + 2 * k] * x0 + sW[kOW1 + 2 * k + 1] * x1 + sW[kOB1 + k];
    sDZ1[tid * kLd + k] = dh * dsilu_f(z1);
  }
  __syncthreads();
  // block partial gradients, samples summed in index order
  float* out = partials + (int64_t)blockIdx.x * kNParam;
  for (int e = tid; e < kNParam; e += kBT) {
    float acc = 0.0f;
    if (e < kOB1) {
      const int k = (e - kOW1) >> 1, c = (e - kOW1) & 1;
      for (int i = 0; i < kBT; ++i) acc += sDZ1[i * kLd + k] * sX[2 * i + c];
    } else if (e < kOW2) {
      const int k = e - kOB1;
      for (int i = 0; i < kBT; ++i) acc += sDZ1[i * kLd + k];
    } else if (e < kOB2) {
      const int j = (e - kOW2) / kH, k = (e - kOW2) % kH;
      for (int i = 0; i < kBT; ++i) acc += sDZ2[i * kLd + j] * sH1[i * kLd + k];
    } else if (e < kOW3) {
      const int j = e - kOB2;
      for (int i = 0; i < kBT; ++i) acc += sDZ2[i * kLd + j];
    } else if (e < kOB3) {
      const int o = (e - kOW3) / kH, j = (e - kOW3) % kH;
      for (int i = 0; i < kBT; ++i) acc += sD[2 * i + o] * silu_exact(sZ2[i * kLd + j]);
    } else {
      const int o = e - kOB3;
      for (int i = 0; i < kBT; ++i) acc += sD[2 * i + o];
    }
    out[e] = acc;
  }
  if (tid == 0) {
    float l = 0.0f;
    for (int i = 0; i < kBT; ++i) l += sL[i];
    loss_partials[blockIdx.x] = l;
  }
}

__global__ void grad_reduce_kernel(const float* __restrict__ partials, int nblocks, const float* __restrict__ loss_partials,
                                   float* __restrict__ grad, float* __restrict__ loss) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kNParam) {
    float acc = 0.0f;
    for (int b = 0; b < nblocks; ++b) acc += partials[(int64_t)b * kNParam + e];
    grad[e] = acc;
  }
  if (e == 0) {
    float l = 0.0f;
    for (int b = 0; b < nblocks; ++b) l += loss_partials[b];
    *loss = l;
  }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1t, float b2t) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParam) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mm = b1 * m[e] + (1.0f - b1) * g[e];
  const float vv = b2 * v[e] + (1.0f - b2) * g[e] * g[e];
  m[e] = mm;
  v[e] = vv;
  const float mh = mm / (1.0f - b1t), vh = vv / (1.0f - b2t);
  p[e] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void eval_kernel(MlpParams W, const double* __restrict__ n, const double* __restrict__ e, int64_t count,
                            double* __restrict__ T, double* __restrict__ mu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float y0, y1, t, m;
  const double delta = 1.5 - 1.5 * e[i] / n[i];
  mlp_forward_f(W, (float)n[i], (float)delta, y0, y1);
  mlp_outputs_to_state(y0, y1, t, m);
  T[i] = t;
  mu[i] = m;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes); }
  template <class X>
  X* as() const {
    return (X*)p;
  }
};

#define CKS(call)                      \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) return LBM_ECUDA; \
  } while (0)

lbm_status upload_doubles(const double* src, int64_t count, int on_device, DevBuf& buf, const double** out,
                          cudaStream_t s) {
  if (on_device) {
    *out = src;
    return LBM_OK;
  }
  CKS(buf.alloc(sizeof(double) * count));
  CKS(cudaMemcpyAsync(buf.p, src, sizeof(double) * count, cudaMemcpyHostToDevice, s));
  *out = buf.as<double>();
  return LBM_OK;
}

unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" {

lbm_status lbm_surrogate_targets(const double* n, const double* t, int64_t count, int32_t on_device, float* feat,
                                 float* targ, void* cuda_stream) {
  if (!n || !t || !feat || !targ || count < 1) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevBuf bn, bt, bf, bg;
  const double *dn, *dt;
  if (upload_doubles(n, count, on_device, bn, &dn, s) != LBM_OK) return LBM_ECUDA;
  if (upload_doubles(t, count, on_device, bt, &dt, s) != LBM_OK) return LBM_ECUDA;
  float *df = feat, *dg = targ;
  if (!on_device) {
    CKS(bf.alloc(sizeof(float) * 2 * count));
    CKS(bg.alloc(sizeof(float) * 2 * count));
    df = bf.as<float>();
    dg = bg.as<float>();
  }
  targets_kernel<<<nb(count, 256), 256, 0, s>>>(dn, dt, count, df, dg);
  CKS(cudaGetLastError());
  if (!on_device) {
    CKS(cudaMemcpyAsync(feat, df, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost, s));
    CKS(cudaMemcpyAsync(targ, dg, sizeof(float) * 2 * count, cudaMemcpyDeviceToHost, s));
  }
  CKS(cudaStreamSynchronize(s));
  return LBM_OK;
}

lbm_status lbm_surrogate_loss_grad(const float* params, const float* feat, const float* targ, int64_t count,
                                   float* grad, double* loss, void* cuda_stream) {
  if (!params || !feat || !targ || !grad || count < 1 || count > (1 << 24)) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nblk = (int)nb(count, kBT);
  DevBuf bp, bf, bg, bpart, blp, bgrad, bloss;
  CKS(bp.alloc(sizeof(float) * kNParam));
  CKS(bf.alloc(sizeof(float) * 2 * count));
  CKS(bg.alloc(sizeof(float) * 2 * count));
  CKS(bpart.alloc(sizeof(float) * kNParam * nblk));
  CKS(blp.alloc(sizeof(float) * nblk));
  CKS(bgrad.alloc(sizeof(float) * kNParam));
  CKS(bloss.alloc(sizeof(float)));
  CKS(cudaMemcpyAsync(bp.p, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
  CKS(cudaMemcpyAsync(bf.p, feat, sizeof(float) * 2 * count, cudaMemcpyHostToDevice, s));
  CKS(cudaMemcpyAsync(bg.p, targ, sizeof(float) * 2 * count, cudaMemcpyHostToDevice, s));
  CKS(cudaFuncSetAttribute(fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(float) * kSmTotal));
  fwd_bwd_kernel<<<nblk, kBT, sizeof(float) * kSmTotal, s>>>(bp.as<float>(), bf.as<float>(), bg.as<float>(), 0, count,
                                                              1.0f / (float)count, bpart.as<float>(), blp.as<float>());
  grad_reduce_kernel<<<nb(kNParam, 256), 256, 0, s>>>(bpart.as<float>(), nblk, blp.as<float>(), bgrad.as<float>(),
                                                      bloss.as<float>());
  CKS(cudaGetLastError());
  float l = 0.f;
  CKS(cudaMemcpyAsync(grad, bgrad.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s));
  CKS(cudaMemcpyAsync(&l, bloss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  if (loss) *loss = (double)l / (double)count;
  return LBM_OK;
}

lbm_status lbm_surrogate_train(const double* n, const double* t, int64_t count, const double* n_val,
                               const double* t_val, int64_t count_val, int32_t on_device, const lbm_train_cfg* cfg,
                               float* params, lbm_train_report* rep, void* cuda_stream) {
  if (!n || !t || !params || !cfg || count < kBT || cfg->epochs < 1 || cfg->batch < kBT ||
      cfg->batch % kBT != 0 || !(cfg->lr > 0.0f))
    return LBM_EINVAL;
  if (count_val > 0 && (!n_val || !t_val)) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t0 = std::chrono::steady_clock::now();
  DevBuf bn, bt, bf, bg, bp, bm, bv, bgrad, bpart, blp, bloss;
  const double *dn, *dt;
  if (upload_doubles(n, count, on_device, bn, &dn, s) != LBM_OK) return LBM_ECUDA;
  if (upload_doubles(t, count, on_device, bt, &dt, s) != LBM_OK) return LBM_ECUDA;
  CKS(bf.alloc(sizeof(float) * 2 * count));
  CKS(bg.alloc(sizeof(float) * 2 * count));
  targets_kernel<<<nb(count, 256), 256, 0, s>>>(dn, dt, count, bf.as<float>(), bg.as<float>());
  const int nblk = cfg->batch / kBT;
  CKS(bp.alloc(sizeof(float) * kNParam));
  CKS(bm.alloc(sizeof(float) * kNParam));
  CKS(bv.alloc(sizeof(float) * kNParam));
  CKS(bgrad.alloc(sizeof(float) * kNParam));
  CKS(bpart.alloc(sizeof(float) * kNParam * nblk));
  CKS(blp.alloc(sizeof(float) * nblk));
  CKS(bloss.alloc(sizeof(float)));
  CKS(cudaMemcpyAsync(bp.p, params, sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
  CKS(cudaMemsetAsync(bm.p, 0, sizeof(float) * kNParam, s));
  CKS(cudaMemsetAsync(bv.p, 0, sizeof(float) * kNParam, s));
  CKS(cudaFuncSetAttribute(fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(float) * kSmTotal));
  const int64_t per_epoch = count / cfg->batch;
  const int64_t total = per_epoch * cfg->epochs;
  const float lr_final = cfg->lr_final > 0.0f ? cfg->lr_final : cfg->lr * 0.01f;
  double b1t = 1.0, b2t = 1.0;
  float first = -1.f, last = -1.f;
  int64_t it = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    for (int64_t b = 0; b < per_epoch; ++b, ++it) {
      fwd_bwd_kernel<<<nblk, kBT, sizeof(float) * kSmTotal, s>>>(bp.as<float>(), bf.as<float>(), bg.as<float>(),
                                                                  b * cfg->batch, cfg->batch, 1.0f / cfg->batch,
                                                                  bpart.as<float>(), blp.as<float>());
      grad_reduce_kernel<<<nb(kNParam, 256), 256, 0, s>>>(bpart.as<float>(), nblk, blp.as<float>(),
                                                          bgrad.as<float>(), bloss.as<float>());
      b1t *= 0.9;
      b2t *= 0.999;
      const double frac = total > 1 ? (double)it / (double)(total - 1) : 1.0;
      const float lr = lr_final + 0.5f * (cfg->lr - lr_final) * (1.0f + (float)cos(kPi * frac));
      adam_kernel<<<nb(kNParam, 256), 256, 0, s>>>(bp.as<float>(), bm.as<float>(), bv.as<float>(), bgrad.as<float>(),
                                                   lr, (float)b1t, (float)b2t);
      if (it == 0) {
        CKS(cudaMemcpyAsync(&first, bloss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
        CKS(cudaStreamSynchronize(s));
      }
    }
  }
  CKS(cudaGetLastError());
  CKS(cudaMemcpyAsync(&last, bloss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
  CKS(cudaMemcpyAsync(params, bp.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  if (rep) {
    rep->iterations = it;
    rep->loss_first = first / cfg->batch;
    rep->loss_last = last / cfg->batch;
    rep->val_rmse_lnT = rep->val_rmse_mu = rep->val_max_rel_x = -1.0;
    if (count_val > 0) {
      DevBuf vn, vt, vf, vg, vT, vmu;
      const double *dvn, *dvt;
      if (upload_doubles(n_val, count_val, on_device, vn, &dvn, s) != LBM_OK) return LBM_ECUDA;
      if (upload_doubles(t_val, count_val, on_device, vt, &dvt, s) != LBM_OK) return LBM_ECUDA;
      CKS(vf.alloc(sizeof(float) * 2 * count_val));
      CKS(vg.alloc(sizeof(float) * 2 * count_val));
      targets_kernel<<<nb(count_val, 256), 256, 0, s>>>(dvn, dvt, count_val, vf.as<float>(), vg.as<float>());
      std::vector<float> f(2 * count_val), gt(2 * count_val);
      CKS(cudaMemcpyAsync(f.data(), vf.p, sizeof(float) * 2 * count_val, cudaMemcpyDeviceToHost, s));
      CKS(cudaMemcpyAsync(gt.data(), vg.p, sizeof(float) * 2 * count_val, cudaMemcpyDeviceToHost, s));
      // network prediction on the validation set (same eval kernel as lbm_surrogate_eval)
      std::vector<double> hn(count_val), he(count_val);
      CKS(cudaStreamSynchronize(s));
      for (int64_t i = 0; i < count_val; ++i) {
        hn[i] = (double)f[2 * i] * kSurNHalf + kSurNMid;
        const double delta = std::exp((double)f[2 * i + 1] * kSurLdHalf + kSurLdMid);
        he[i] = hn[i] * (1.5 - delta) / 1.5;
      }
      DevBuf dn2, de2;
      CKS(dn2.alloc(sizeof(double) * count_val));
      CKS(de2.alloc(sizeof(double) * count_val));
      CKS(vT.alloc(sizeof(double) * count_val));
      CKS(vmu.alloc(sizeof(double) * count_val));
      CKS(cudaMemcpyAsync(dn2.p, hn.data(), sizeof(double) * count_val, cudaMemcpyHostToDevice, s));
      CKS(cudaMemcpyAsync(de2.p, he.data(), sizeof(double) * count_val, cudaMemcpyHostToDevice, s));
      MlpParams W;
      for (int e = 0; e < kNParam; ++e) W.p[e] = params[e];
      eval_kernel<<<nb(count_val, 128), 128, 0, s>>>(W, dn2.as<double>(), de2.as<double>(), count_val,
                                                    vT.as<double>(), vmu.as<double>());
      std::vector<double> T(count_val), mu(count_val);
      CKS(cudaMemcpyAsync(T.data(), vT.p, sizeof(double) * count_val, cudaMemcpyDeviceToHost, s));
      CKS(cudaMemcpyAsync(mu.data(), vmu.p, sizeof(double) * count_val, cudaMemcpyDeviceToHost, s));
      CKS(cudaStreamSynchronize(s));
      double sl = 0, sm = 0, mx = 0;
      for (int64_t i = 0; i < count_val; ++i) {
        const double lnT_true = (double)gt[2 * i] * kSurLnTHalf + kSurLnTMid;
        const double mu_true = (double)gt[2 * i + 1] * kSurMuHalf + kSurMuMid;
        const double dl = std::log(T[i]) - lnT_true, dm = mu[i] - mu_true;
        sl += dl * dl;
        sm += dm * dm;
        const double x_true = mu_true / std::exp(lnT_true), x_pred = mu[i] / T[i];
        mx = std::fmax(mx, std::fabs(x_pred - x_true) / std::fabs(x_true));
      }
      rep->val_rmse_lnT = std::sqrt(sl / count_val);
      rep->val_rmse_mu = std::sqrt(sm / count_val);
      rep->val_max_rel_x = mx;
    }
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return LBM_OK;
}

lbm_status lbm_surrogate_eval(const float* params, const double* n, const double* e, int64_t count, double* T,
                              double* mu, int32_t on_device, void* cuda_stream) {
  if (!params || !n || !e || !T || !mu || count < 1) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevBuf bn, be, bT, bmu;
  const double *dn, *de;
  if (upload_doubles(n, count, on_device, bn, &dn, s) != LBM_OK) return LBM_ECUDA;
  if (upload_doubles(e, count, on_device, be, &de, s) != LBM_OK) return LBM_ECUDA;
  double *dT = T, *dmu = mu;
  if (!on_device) {
    CKS(bT.alloc(sizeof(double) * count));
    CKS(bmu.alloc(sizeof(double) * count));
    dT = bT.as<double>();
    dmu = bmu.as<double>();
  }
  MlpParams W;
  for (int i = 0; i < kNParam; ++i) W.p[i] = params[i];
  eval_kernel<<<nb(count, 128), 128, 0, s>>>(W, dn, de, count, dT, dmu);
  CKS(cudaGetLastError());
  if (!on_device) {
    CKS(cudaMemcpyAsync(T, dT, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    CKS(cudaMemcpyAsync(mu, dmu, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
  }
  return LBM_OK;
}

}  // extern "C"
