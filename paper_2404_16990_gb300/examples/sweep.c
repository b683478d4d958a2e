/*
 * sweep.c -- the C ABI from plain C, without Python: one 256 x 256 lattice at
 * T = 2.269185 from a random start, 1000 checkerboard Metropolis sweeps, E
 * and M read back.  The caller owns the device workspace and the stream.
 *
 * Build after libising.so exists (paper_2404_16990_gb300/build.py):
 *   gcc -std=c99 sweep.c -I../../include -I/usr/local/cuda/include \
 *       -L.. -lising -L/usr/local/cuda/lib64 -lcudart -Wl,-rpath,'$ORIGIN/..' -o sweep
 * (the binary beside this file, so that the rpath finds ../libising.so).  On
 * a GB300 it prints E/N = -1.414001, M/N = 0.020416 (bit-reproducible; the
 * infinite lattice has E/N = -sqrt(2) at T_c).
 */
#include <stdio.h>

#include <cuda_runtime.h>

#include "ising.h"

static int report(const char* what, int rc)
{
    if (rc != ISING_OK) fprintf(stderr, "%s failed (%d): %s\n", what, rc, ising_last_error());
    return rc != ISING_OK;
}

int main(void)
{
    const int L = 256;
    const double T = 2.269185;
    size_t bytes = 0;
    void* workspace = NULL;
    cudaStream_t stream = NULL;
    ising_t h = NULL;
    int64_t E = 0, M = 0;
    int failed = 0;

    if (report("ising_workspace_bytes", ising_workspace_bytes(L, 1, 0, &bytes))) return 1;
    if (cudaStreamCreate(&stream) != cudaSuccess || cudaMalloc(&workspace, bytes) != cudaSuccess) {
        fprintf(stderr, "no CUDA device or out of memory\n");
        return 1;
    }
    failed = report("ising_create",
                    ising_create(&h, L, 1, &T, 1, ISING_INIT_RANDOM, 0, workspace, bytes, (void*)stream));
    if (!failed) failed = report("ising_sweep", ising_sweep(h, 1000));
    if (!failed) failed = report("ising_observables", ising_observables(h, &E, &M));
    if (!failed)
        printf("L=%d T=%.6f after %lld sweeps: E/N = %.6f, M/N = %.6f\n", L, T, (long long)ising_sweeps_done(h),
               (double)E / (L * L), (double)M / (L * L));
    ising_destroy(h);
    cudaFree(workspace);
    cudaStreamDestroy(stream);
    return failed;
}
