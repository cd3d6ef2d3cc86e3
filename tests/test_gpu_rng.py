"""Pins the oracle's Philox4x32-10 (Salmon et al., SC'11) on counter word 3,
which the host-generator pin (test_oracle_philox.py) leaves at zero: cuRAND's
device API, run as a library on the GPU.  curand_init(seed, subsequence,
offset) with offset = 4 b positions the state at block (subsequence, b) of
the seed's stream; curand4 then returns Philox of the counter (b lo32, b hi32,
subsequence lo32, subsequence hi32) under the key (seed lo32, seed hi32).  The
oracle's outputs for those counters must equal cuRAND's, with word 3 (the
chain-group word of the simulation's counters) non-zero."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_SRC = r"""
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void draw(const unsigned long long *seed, const unsigned long long *subseq,
                     const unsigned long long *block, uint4 *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed[i], subseq[i], 4ull * block[i], &st);
  out[i] = curand4(&st);
}

extern "C" int run(const unsigned long long *seed, const unsigned long long *subseq,
                   const unsigned long long *block, uint32_t *out, int n) {
  unsigned long long *d[3];
  uint4 *dout;
  const unsigned long long *h[3] = {seed, subseq, block};
  for (int k = 0; k < 3; k++) {
    if (cudaMalloc(&d[k], n * sizeof(unsigned long long)) != cudaSuccess) return 1;
    cudaMemcpy(d[k], h[k], n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  }
  if (cudaMalloc(&dout, n * sizeof(uint4)) != cudaSuccess) return 1;
  draw<<<(n + 127) / 128, 128>>>(d[0], d[1], d[2], dout, n);
  cudaError_t e = cudaMemcpy(out, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost);
  for (int k = 0; k < 3; k++) cudaFree(d[k]);
  cudaFree(dout);
  return e == cudaSuccess ? 0 : 2;
}
"""


@pytest.fixture(scope="module")
def curand_dev():
    tmp = tempfile.mkdtemp(prefix="pbn_curand_")
    src, so = os.path.join(tmp, "draw.cu"), os.path.join(tmp, "libdraw.so")
    with open(src, "w") as f:
        f.write(_SRC)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.check_call([nvcc, "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-o", so, src])
    return ctypes.CDLL(so)


def test_philox_word3_matches_curand_device(orc, curand_dev):
    rng = np.random.default_rng(3)
    n = 64
    seed = rng.integers(0, 1 << 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n).astype(np.uint64)
    subseq = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    subseq[:8] = [1 << 32, 5 << 32, (7 << 32) | 3, 0xFFFFFFFF << 32, 1, 2, 0, (1 << 40) | 9]
    block = rng.integers(0, 1 << 40, size=n, dtype=np.uint64)
    out = np.zeros(4 * n, dtype=np.uint32)
    p = ctypes.c_void_p
    rc = curand_dev.run(p(seed.ctypes.data), p(subseq.ctypes.data), p(block.ctypes.data), p(out.ctypes.data),
                        ctypes.c_int(n))
    assert rc == 0
    assert np.count_nonzero(subseq >> np.uint64(32)) >= n // 2
    for i in range(n):
        s, q, b = int(seed[i]), int(subseq[i]), int(block[i])
        ctr = [b & 0xFFFFFFFF, b >> 32, q & 0xFFFFFFFF, q >> 32]
        mine = orc.philox4x32_10(ctr, [s & 0xFFFFFFFF, s >> 32])
        assert list(mine) == list(out[4 * i:4 * i + 4]), i
