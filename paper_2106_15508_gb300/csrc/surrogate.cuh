// surrogate.cuh -- parameter layout and state of the MLP surrogate.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "../../include/abcsmc.h"

namespace abc {

constexpr int kMlpH = 256;                                // hidden width
constexpr int kOffW1 = 0;                                 // W1[256][8]
constexpr int kOffB1 = kOffW1 + kMlpH * 8;                // b1[256]
constexpr int kOffW2 = kOffB1 + kMlpH;                    // W2[256][256]
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;            // b2[256]
constexpr int kOffW3 = kOffB2 + kMlpH;                    // W3[4][256]
constexpr int kOffB3 = kOffW3 + 4 * kMlpH;                // b3[4]
constexpr int kMlpParams = kOffB3 + 4;                    // 69124 parameters
constexpr uint32_t kTagMlpInit = 9;                       // Philox stream of the initial weights
constexpr uint32_t kTagScreen = ABC_TAG_SCREEN;           // screening uniforms (delayed acceptance)
constexpr uint32_t kTagAudit = ABC_TAG_AUDIT;             // audit uniforms of screened-out proposals
constexpr uint32_t kTagTrain = 10;                        // minibatch indices

struct MlpState {
  float* w;              // fp32 master parameters
  __nv_bfloat16* wb;     // bf16 copy used by every product
  float* m;              // Adam first moments
  float* v;              // Adam second moments
};

// host entry points (surrogate.cu)
int mlp_init(const MlpState& s, uint32_t k0, uint32_t k1, cudaStream_t st);
int mlp_refresh_bf16(const MlpState& s, cudaStream_t st);
size_t mlp_train_scratch_bytes(int B);
int mlp_grad(const MlpState& s, const float* X, const float* T, int B, float* grad, float* loss_dev,
             void* scratch, size_t bytes, cudaStream_t st, unsigned* err = nullptr);
unsigned* mlp_grad_err(void* scratch, int B);
int mlp_train_prepare();
int mlp_adam(const MlpState& s, const float* grad, int64_t step, float lr, cudaStream_t st);
size_t mlp_infer_scratch_bytes(int64_t n);
int mlp_infer_prepare();
unsigned* mlp_infer_err(void* scratch, int64_t n);
int mlp_infer(const MlpState& s, const float* u, int64_t n, float* Y, void* scratch, size_t bytes,
              unsigned** err_out, cudaStream_t st, bool reset_err = true,
              unsigned* err_word = nullptr, const float* xstat = nullptr);
size_t screen_scratch_bytes(int64_t M);
int screen(const float* Y, const float* ystat, const uint8_t* pflag, int64_t M, const double* eps,
           uint32_t k0, uint32_t k1, uint32_t c1, float tau, float rho_min, float audit_frac,
           float* rho, uint8_t* sflag, cudaStream_t st, unsigned long long* exhausted,
           const uint32_t* c1_dev = nullptr, const int* on_dev = nullptr);
int screen_and_compact(const float* Y, const float* ystat, const uint8_t* pflag, int64_t M,
                       const double* eps, uint32_t k0, uint32_t k1, uint32_t c1, float tau,
                       float rho_min, float audit_frac, float* rho, uint8_t* sflag,
                       const float* up, const float* sp, const int32_t* ap, float* cu, float* cs,
                       int32_t* ca, float* crho, uint8_t* cflag, uint32_t* cslot, int* Mc_dev,
                       void* scratch, cudaStream_t st, unsigned long long* exhausted,
                       const uint32_t* c1_dev, const int* on_dev, long long* sim_acc);
size_t ring_scratch_bytes(int64_t n);
int ring_append(const uint8_t* invalid, int64_t n, const float* u, const double* d,
                const int32_t* ard, long long* head, int64_t cap, float* RX, float* RY,
                void* scratch, cudaStream_t st, const int* n_dev = nullptr);
// ystat [24]: output means [4] and standard deviations [4], then input means
// [8] and standard deviations [8], over the filled ring
// ystat before any training: means 0, standard deviations 1
int stats_init(float* ystat, cudaStream_t st);
int ring_stats(const float* RX, const float* RY, const long long* head, int64_t cap, float* ystat,
               void* scratch, cudaStream_t st);
size_t ring_stats_scratch_bytes();
int mlp_train(const MlpState& s, const float* RX, const float* RY, const long long* head,
              int64_t cap, const float* ystat, int B, int steps, uint32_t* step_dev, float lr,
              uint32_t k0, uint32_t k1, float* grad, float* X, float* T, float* loss_dev,
              void* scratch, size_t bytes, cudaStream_t st, const int* off_dev = nullptr,
              unsigned* err = nullptr);
int sur_gate(const uint32_t* t_dev, uint32_t t, int start, const uint32_t* step_dev, int* on,
             cudaStream_t st);
int audit_count(const uint8_t* cflag, const double* cd, const int* Mc, const double* eps,
                unsigned long long* counts, cudaStream_t st);
int rho_correct(double* logW, const float* rho, int64_t n, cudaStream_t st,
                const int* off_dev = nullptr);

}  // namespace abc
