"""The rule that decides which caller buffers the allocation-free Lloyd step
may hand to its kernels (paper_2506_03437_b300/csrc/devmem.h), checked on the
host: a small C++ program built with g++ against the CUDA headers feeds it
pointer attributes of every kind, so no GPU and no launch is involved.
Memory of another GPU must be refused, since the library enables no peer
access and a kernel given such a pointer faults."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2506_03437_b300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

PROGRAM = r"""
#include <cstdio>
#include <cstring>
#include "devmem.h"
static cudaPointerAttributes attr(cudaMemoryType t, int dev) {
  cudaPointerAttributes a;
  std::memset(&a, 0, sizeof(a));
  a.type = t;
  a.device = dev;
  return a;
}
int main() {
  // current device 1 of several
  std::printf("%d %d %d %d %d %d\n",
              (int)qk::usable_on_device(attr(cudaMemoryTypeDevice, 1), 1),
              (int)qk::usable_on_device(attr(cudaMemoryTypeDevice, 0), 1),
              (int)qk::usable_on_device(attr(cudaMemoryTypeDevice, 2), 1),
              (int)qk::usable_on_device(attr(cudaMemoryTypeManaged, 0), 1),
              (int)qk::usable_on_device(attr(cudaMemoryTypeHost, 1), 1),
              (int)qk::usable_on_device(attr(cudaMemoryTypeUnregistered, 0), 1));
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime_api.h")),
                    reason="needs g++ and the CUDA headers")
def test_only_this_gpus_memory_or_managed_memory_is_usable(tmp_path):
    src = tmp_path / "devmem_check.cpp"
    exe = tmp_path / "devmem_check"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    # own device memory yes; other GPUs' no; managed yes; pinned and plain host memory no
    assert out == ["1", "0", "0", "1", "0", "0"]
