"""The library's host routine for the rotational primal constraints
(csrc/rigid.h: principal axes of the class by cyclic Jacobi, rows
v x (x - xbar) / sqrt(moment)) against the oracle's (SVD of the three
rotation fields): same number of rows, orthonormal rows, the same span, on
random clouds over several scales, straight lines (axial rotation dropped),
planar sets, a square (repeated principal moments) and single nodes.
Compiled for the host with g++ here; no GPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.bddc import class_rotations

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WRAPPER = r"""
#include "rigid.h"
#include <cstring>
extern "C" int rotations(const double* X, int m, double* out) {
  std::vector<double> x(X, X + 3 * (size_t)m);
  std::vector<int> nodes(m);
  for (int i = 0; i < m; ++i) nodes[i] = i;
  std::vector<double> w;
  const int n = cbddc::class_rotations(x, nodes, w);
  if (!w.empty()) std::memcpy(out, w.data(), w.size() * sizeof(double));
  return n;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("rigid")
    src = d / "wrap.cpp"
    src.write_text(WRAPPER)
    so = d / "librigid.so"
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2208_06191_gb300", "csrc"), str(src), "-o", str(so)],
                   check=True, capture_output=True)
    return ctypes.CDLL(str(so))


def _lib_rows(lib, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(9 * len(X))
    n = lib.rotations(X.ctypes.data_as(ctypes.c_void_p), len(X), out.ctypes.data_as(ctypes.c_void_p))
    return out[:3 * len(X) * n].reshape(n, 3 * len(X))


def _cases():
    rng = np.random.default_rng(0)
    cases = [rng.standard_normal((m, 3)) * rng.uniform(1e-3, 10.0) + rng.standard_normal(3)
             for m in range(2, 30)]
    for m in (2, 3, 7):
        cases.append(np.c_[np.linspace(0.0, 1.0, m), np.zeros(m), np.zeros(m)] + 0.3)
    t = rng.standard_normal(3)
    t /= np.linalg.norm(t)
    cases.append(np.outer(np.linspace(-1.0, 1.0, 5), t) + 2.0)
    cases.append(np.c_[rng.uniform(size=(9, 2)), np.full(9, 0.7)])
    cases.append(np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0], [1.0, 1, 0]]))
    cases.append(np.array([[0.1, 0.2, 0.3]]))
    return cases


@pytest.mark.parametrize("k", range(len(_cases())))
def test_library_rotations_match_oracle(lib, k):
    X = _cases()[k]
    A = _lib_rows(lib, X)
    B = class_rotations(X)
    assert A.shape == B.shape
    if A.shape[0] == 0:
        return
    assert np.abs(A @ A.T - np.eye(A.shape[0])).max() <= 1e-12
    assert np.linalg.norm(B - B @ A.T @ A) <= 1e-12 * np.sqrt(A.shape[0])
