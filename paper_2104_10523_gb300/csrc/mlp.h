// Learned path cost model (see mlp.cu): device state and host entry points.
#pragma once

#include <cstdint>
#include <vector>

#include "executor.h"

namespace tnq {

constexpr int kStepFeatures = 16;

struct CostModel {
  int d_in = kStepFeatures, h = 256, max_batch = 4096;
  uint64_t seed = 0;
  std::vector<float> host_params;  // FP32 master weights W1 b1 W2 b2 W3 b3 (flat)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  long adam_t = 0;
  // workspace offsets (bytes)
  size_t o_params = 0, o_grads = 0, o_m = 0, o_v = 0, o_w1b = 0, o_w2b = 0, o_w3b = 0, o_x = 0, o_t = 0, o_z1 = 0,
         o_a1 = 0, o_z2 = 0, o_a2 = 0, o_y = 0, o_dy = 0, o_sq = 0, o_dz1 = 0, o_dz2 = 0, o_loss = 0;
  size_t n_params() const;
  void layout();
};

void mlp_init(CostModel* m);
tnq_status mlp_bind(Ctx* ctx, CostModel* m, void* ws, size_t bytes);
tnq_status mlp_upload(Ctx* ctx, CostModel* m, const float* params);
tnq_status mlp_download(Ctx* ctx, CostModel* m, float* params);
tnq_status mlp_gradients(Ctx* ctx, CostModel* m, const float* X, const float* t, int64_t n, float* grads, float* loss);
tnq_status mlp_train(Ctx* ctx, CostModel* m, const float* X, const float* t, int64_t n, int epochs, int batch,
                     float lr, float* final_loss);
tnq_status mlp_predict(Ctx* ctx, CostModel* m, const float* X, int64_t n, float* y);

// Features of every step of a laid-out plan, for the kernels `precision` dispatches to.
void step_features(const Plan& p, int precision, std::vector<float>* out);

}  // namespace tnq

struct tnq_cost_model { tnq::CostModel m; };
