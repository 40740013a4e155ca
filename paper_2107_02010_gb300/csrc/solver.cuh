// Internal interface between the C-ABI layer (solver.cu) and the solve
// routines (sinkhorn.cu, multiscale.cu, transport.cu).
#pragma once

#include <vector>

#include "otgb_internal.cuh"

namespace otgb {

std::vector<double> make_schedule(double d, double blur, double q);
// lambda = 1 / (1 + (sigma / reach)^p), the unbalanced damping of the Algorithm (Section 2); 1 when balanced
double lambda_of(double sigma, double reach, int p = 2);

int fail(otgb_ctx *ctx, const Error &e);
cudaStream_t ctx_stream(otgb_ctx *ctx);
Workspace &ctx_ws(otgb_ctx *ctx);
void *ctx_pinned(otgb_ctx *ctx);
cudaEvent_t ctx_event(otgb_ctx *ctx, int k);
void ctx_set_device(otgb_ctx *ctx);
int ctx_sm_count(otgb_ctx *ctx);

}  // namespace otgb
