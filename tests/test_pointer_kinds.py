"""The library's decision about a caller buffer from cudaPointerGetAttributes'
answer (csrc/pointers.h): host memory is copied, memory of the call's device
or managed memory is used in place, and device memory of another GPU is
rejected before any kernel sees it.  The predicate is compiled on the host
and checked on its truth table; no buffer is handed to a kernel."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_20176_b300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cstdio>
#include "pointers.h"
using snaps::PtrKind;
using snaps::ptr_kind_of;
int main() {
    int bad = 0;
    auto expect = [&](cudaMemoryType t, int owner, int dev, PtrKind want) {
        if (ptr_kind_of(t, owner, dev) != want) { std::printf("fail %d %d %d\n", (int)t, owner, dev); ++bad; }
    };
    expect(cudaMemoryTypeUnregistered, -2, 0, PtrKind::Host);
    expect(cudaMemoryTypeHost, 0, 0, PtrKind::Host);
    expect(cudaMemoryTypeHost, 1, 0, PtrKind::Host);
    expect(cudaMemoryTypeDevice, 0, 0, PtrKind::Device);
    expect(cudaMemoryTypeDevice, 3, 3, PtrKind::Device);
    expect(cudaMemoryTypeDevice, 1, 0, PtrKind::Foreign);
    expect(cudaMemoryTypeDevice, 0, 7, PtrKind::Foreign);
    expect(cudaMemoryTypeManaged, 0, 0, PtrKind::Device);
    expect(cudaMemoryTypeManaged, 2, 5, PtrKind::Device);
    std::printf("%s\n", bad ? "BAD" : "OK");
    return bad;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC),
                    reason="needs g++ and the CUDA headers")
def test_pointer_kind_truth_table(tmp_path):
    src = tmp_path / "kinds.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "kinds"
    subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout
