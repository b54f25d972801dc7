"""Grouped accumulation of psi (Eq. U_1) in the single-order launches, checked on the host.

The launch forming T_k adds to the accumulator only when k = 2 (mod 3) or k = M, and then adds
the orders formed since the previous such launch.  The schedule (AccGroup in the library's
internal header) is compiled here as a host program and run for every truncation order
M <= 60 and every complex64 split: each order 0..M must be added exactly once, to psi when it
is <= ksplit and to the tail accumulator otherwise, each accumulator must be read exactly when
an earlier group has written it, and the last launch must combine psi and the tail.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_0907_3022_gb300", "csrc")

PROGRAM = r'''
#include "cheb_internal.cuh"
#include <algorithm>
#include <cstdio>
#include <set>
using namespace cheb;
int main() {
    int bad = 0;
    for (int M = 2; M <= 60; ++M) {
        for (int k0 = 2; k0 <= 70; ++k0) {
            const int ks = std::min(k0 + ((2 - k0 % 3) + 3) % 3, M);  // as the plan sets it
            std::set<int> psi, tail;
            bool psi_has = false, tail_has = false, done = false;
            for (int k = 1; k <= M; ++k) {
                const AccGroup ag(k, M, ks);
                if (!ag.upd) continue;
                if (ag.read_acc != (ag.to_tail ? tail_has : psi_has)) bad++;
                const int first = (k == 2) ? 0 : k - ag.n + 1;
                if (ag.n < 1 || ag.n > 3 || (k == 2 && ag.n != 3)) bad++;
                for (int o = first; o <= k; ++o) {
                    if (psi.count(o) || tail.count(o)) bad++;
                    (ag.to_tail ? tail : psi).insert(o);
                    if (ag.to_tail != (o > ks)) bad++;
                }
                (ag.to_tail ? tail_has : psi_has) = true;
                if (ag.last) {
                    done = true;
                    if (ag.read_psi_last != ag.to_tail) bad++;
                }
            }
            if (!done || (int)(psi.size() + tail.size()) != M + 1) bad++;
        }
    }
    printf("bad=%d\n", bad);
    return bad != 0;
}
'''


def test_accumulation_schedule(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "accg.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "accg"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True,
                   capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and "bad=0" in r.stdout, r.stdout + r.stderr
