"""The oracle's Philox4x32-10 against cuRAND's device function
curand_Philox4x32_10 (called from a kernel compiled here, not copied), on
counters with all four words non-zero and arbitrary keys."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

KERNEL = r"""
#include <cstdio>
#include <curand_kernel.h>
__global__ void k(const uint4 *c, const uint2 *key, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(c[i], key[i]);
}
int main() {
    const int n = 64;
    uint4 hc[n], ho[n]; uint2 hk[n];
    unsigned s = 12345u;
    auto nx = [&]() { s = s * 1664525u + 1013904223u; return s; };
    for (int i = 0; i < n; ++i) { hc[i] = make_uint4(nx(), nx(), nx(), nx()); hk[i] = make_uint2(nx(), nx()); }
    uint4 *dc, *dout; uint2 *dk;
    cudaMalloc(&dc, sizeof(hc)); cudaMalloc(&dk, sizeof(hk)); cudaMalloc(&dout, sizeof(ho));
    cudaMemcpy(dc, hc, sizeof(hc), cudaMemcpyHostToDevice);
    cudaMemcpy(dk, hk, sizeof(hk), cudaMemcpyHostToDevice);
    k<<<1, 64>>>(dc, dk, dout, n);
    if (cudaMemcpy(ho, dout, sizeof(ho), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    for (int i = 0; i < n; ++i)
        printf("%u %u %u %u %u %u %u %u %u %u\n", hc[i].x, hc[i].y, hc[i].z, hc[i].w, hk[i].x, hk[i].y,
               ho[i].x, ho[i].y, ho[i].z, ho[i].w);
    return 0;
}
"""


def test_oracle_philox_matches_curand_device_function():
    require_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "kat.cu")
        exe = os.path.join(td, "kat")
        with open(src, "w") as f:
            f.write(KERNEL)
        subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = [list(map(int, l.split())) for l in out.strip().splitlines()]
    assert len(rows) == 64
    for r in rows:
        assert all(v != 0 for v in r[:4])
        got = oracle.philox4x32_10(r[0:4], r[4:6])
        assert np.array_equal(got, np.array(r[6:10], np.uint32)), r
