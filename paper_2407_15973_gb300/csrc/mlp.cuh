// Learned per-block format selector: a 12 -> 64 -> 64 -> 3 ReLU MLP over block features.
#pragma once
#include "common.cuh"

namespace mpbjac {

constexpr int kFeat = 12, kH1 = 64, kH2 = 64, kCls = 3;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kH1 * kFeat;
constexpr int kOffW2 = kOffB1 + kH1;
constexpr int kOffB2 = kOffW2 + kH2 * kH1;
constexpr int kOffW3 = kOffB2 + kH2;
constexpr int kOffB3 = kOffW3 + kCls * kH2;
constexpr int kMlpWeights = kOffB3 + kCls;          // 5187 trainable parameters
constexpr int kOffMu = kMlpWeights;
constexpr int kOffSd = kOffMu + kFeat;
constexpr int kMlpParams = kOffSd + kFeat;          // + feature mean and standard deviation

// params: HOST floats [kMlpParams]. Writes fmt[b] for every block (class -> format, then
// promotion until kappa_1 * u_f <= safety_theta).
// The forward pass runs on the tensor cores (tcgen05); a tile whose MMA does not complete in
// the bounded wait leaves fmt 0xFF for its blocks (the caller reports a timeout).
int launch_mlp_select(const float *params, int nb, const double *feat, const double *kap, double safety_theta,
                      uint8_t *fmt, cudaStream_t st);
// logits[3 n] of the same tensor-core forward pass (dparams: DEVICE floats [kMlpParams]);
// entries of a tile whose MMA timed out are NaN
int launch_mlp_logits_tc(const float *dparams, int n, const double *feat, float *logits, cudaStream_t st);
// Gradient of the loss sum / N over N samples with the weights rounded to bfloat16, layer 2's
// three products on the tensor cores: CTA c of `grid` (mlp_grad_tc_grid(N)) writes its partial
// gradient to partial[c][kMlpWeights] and its loss sum to loss_part[c] (NaN after an MMA that
// did not complete in the bounded wait)
int mlp_grad_tc_grid(int N);
int launch_mlp_grad_tc(const float *dparams, const double *feat, const int32_t *label, int N, float *partial,
                       double *loss_part, int grid, cudaStream_t st);

}  // namespace mpbjac
