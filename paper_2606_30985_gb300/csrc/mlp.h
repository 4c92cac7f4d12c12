// Internal API of the learned BP warm start (k_mlp.cu).
#pragma once
#include "common.cuh"

#ifndef PEPO_WS_FEATURES
#define PEPO_WS_FEATURES 12
#define PEPO_WS_WIDTH 256
#endif

namespace pepo {

// static description of one directed bond for the feature rows
struct WsGeom {
  int n_other;          // other bonds at the source site (<= 3)
  int other[3];
  float deg_src, deg_dst;     // site degrees
  float dist_src, dist_dst;   // Manhattan distance to the observable / (Lx + Ly)
};

struct MlpBuffers {
  float *p, *m, *v, *g, *pr;           // master params, Adam moments, gradient, BF16-rounded params
  float *x, *z1, *a1, *z2, *a2, *y, *dy, *d2, *d1, *loss;
};

long long mlp_num_params();
// carves the buffers from base (nullptr: size only); returns the bytes needed
size_t mlp_layout(char* base, int max_rows, MlpBuffers* B);
cudaError_t mlp_forward(const MlpBuffers& B, const float* X, int rows, float* y_out, cudaStream_t s);
cudaError_t mlp_gradient(const MlpBuffers& B, const float* X, const float* t, int rows, cudaStream_t s);
cudaError_t mlp_adam(const MlpBuffers& B, int t, float lr, cudaStream_t s);

cudaError_t launch_ws_features(const WsGeom* geom, int nb, const int* chi, const double* lam, int ldl, float t,
                               float h, float J, float* X, int max_rows, cudaStream_t s);
cudaError_t launch_ws_targets(int nb, const int* chi, const double* msg, int ldm, float* out, int max_rows,
                              cudaStream_t s);
cudaError_t launch_ws_apply(int nb, const int* chi, const float* y, double* msg, int ldm, float gamma,
                            cudaStream_t s);

}  // namespace pepo
