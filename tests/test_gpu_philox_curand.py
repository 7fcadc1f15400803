"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11; the keyed randomness
that stands for the paper's hash of (j, k, t), Sec. 3.2) pinned on the device
against NVIDIA's implementation: a small program built at test time calls the
cuRAND header's Philox4x32-10 block function for the same (counter, key)
pairs, and its blocks must equal the oracle's.  This pin needs no Python
package, only the CUDA toolkit and a GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

_PROGRAM = r"""
#include <cstdio>
#include <curand_philox4x32_x.h>

__global__ void blocks(const uint4* c, const uint2* k, uint4* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(c[i], k[i]);
}

int main() {
    int n = 0;
    if (scanf("%d", &n) != 1 || n <= 0 || n > 4096) return 2;
    uint4 hc[4096];
    uint2 hk[4096];
    for (int i = 0; i < n; ++i)
        if (scanf("%x %x %x %x %x %x", &hc[i].x, &hc[i].y, &hc[i].z, &hc[i].w, &hk[i].x, &hk[i].y) != 6) return 2;
    uint4 *dc, *dout;
    uint2* dk;
    if (cudaMalloc(&dc, n * sizeof(uint4)) || cudaMalloc(&dk, n * sizeof(uint2)) || cudaMalloc(&dout, n * sizeof(uint4)))
        return 3;
    cudaMemcpy(dc, hc, n * sizeof(uint4), cudaMemcpyHostToDevice);
    cudaMemcpy(dk, hk, n * sizeof(uint2), cudaMemcpyHostToDevice);
    blocks<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
    uint4 ho[4096];
    if (cudaMemcpy(ho, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
    for (int i = 0; i < n; ++i) printf("%08x %08x %08x %08x\n", ho[i].x, ho[i].y, ho[i].z, ho[i].w);
    return 0;
}
"""


def _nvcc():
    for cand in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


@pytest.mark.gpu
def test_philox_matches_curand_header(tmp_path, oracle):
    rng = np.random.default_rng(2011)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2), ([1, 2, 3, 4], [5, 6])]
    for _ in range(500):
        cases.append((rng.integers(0, 2**32, size=4).tolist(), rng.integers(0, 2**32, size=2).tolist()))
    # the counters the samplers use: (block t, tag, node id lo, node id hi)
    for tag in range(1, 7):
        for t in (0, 1, 1000, 2**32 - 1):
            node = int(rng.integers(1, 2**40))
            seed = int(rng.integers(0, 2**64, dtype=np.uint64))
            cases.append(([t, tag, node & 0xFFFFFFFF, node >> 32], [seed & 0xFFFFFFFF, seed >> 32]))
    src = tmp_path / "philox_curand.cu"
    exe = tmp_path / "philox_curand"
    src.write_text(_PROGRAM)
    subprocess.run([_nvcc(), "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(exe), str(src)],
                   check=True, capture_output=True, text=True)
    inp = f"{len(cases)}\n" + "".join(" ".join(f"{int(x):x}" for x in c + k) + "\n" for c, k in cases)
    p = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    lines = p.stdout.strip().splitlines()
    assert len(lines) == len(cases)
    for (c, k), line in zip(cases, lines):
        assert oracle.philox4x32_10(c, k) == [int(w, 16) for w in line.split()], (c, k)
