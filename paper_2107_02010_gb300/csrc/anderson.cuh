// Anderson acceleration of the Sinkhorn fixed-point map (anderson.cu).
#pragma once

#include <string>

#include "otgb_internal.cuh"

namespace otgb {

constexpr int kAAMax = 8;  // longest history (differences)

struct Anderson {
    int n = 0, m = 0, slots = 0;
    double reg = 1e-9;         // Tikhonov weight relative to the mean diagonal of the normal matrix
    float *Rring = nullptr, *Gring = nullptr;
    double *part = nullptr, *Q = nullptr, *coef = nullptr, *best = nullptr;
    int *state = nullptr;      // device: newest slot, valid entries, restarts
    void init(Workspace &ws, const std::string &tag, int n, int m, cudaStream_t st);
    void reset(cudaStream_t st);
    // z: the iterate the step started from; G: its image G(z), overwritten by z_{k+1}
    void step(const float *z, float *G, cudaStream_t st);
};

}  // namespace otgb
