// Family E launchers (kern_1dflux.cu): Burgers IC + mass + Godunov flux rows.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "snap_internal.h"

size_t ws_bytes_1dflux(const snap_problem *p, int B);
cudaError_t launch_1dflux_forward(const snap_problem *p, int B, const double *u_hat,
                                  const double *params, double *u, double *lambda,
                                  snap_stats *stats, const SolverOpts &o, void *ws,
                                  cudaStream_t s);
cudaError_t launch_1dflux_backward(const snap_problem *p, int B, const double *grad_u,
                                   const double *u, const snap_stats *stats, double *grad_u_hat,
                                   double *grad_params, void *ws, cudaStream_t s);
cudaError_t launch_1dflux_residual(const snap_problem *p, int B, const double *u,
                                   const double *params, double *h, double *h_inf, void *ws,
                                   cudaStream_t s);
