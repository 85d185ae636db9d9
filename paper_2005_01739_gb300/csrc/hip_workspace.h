// Per-device scratch owned by the library: one device buffer that grows on
// demand (never shrinks) and is carved into 256-byte aligned pieces per call.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/hipster_gb300.h"

struct Workspace {
    void *base = nullptr;
    size_t cap = 0;
    hip_status reserve(size_t bytes, cudaStream_t st);
};

struct Carve {
    size_t total = 0;
    size_t take(size_t bytes)
    {
        size_t off = total;
        total += (bytes + 255) & ~(size_t)255;
        return off;
    }
};

Workspace &hip_workspace(int dev);
// The message hip_last_error() returns: cleared at the start of a public call,
// set with the failing step and the CUDA error when one fails.
void hip_clear_error();
void hip_set_error(const char *what, cudaError_t e);
hip_status hip_device_setup(int *dev_out);
bool hip_is_device_ptr(const void *p);
int hip_cells_per_side(double L, double R0);
hip_status hip_check_edges(const double *k_edges, int n_k);
