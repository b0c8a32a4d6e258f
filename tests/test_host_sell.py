"""The library's host routine that lays out the BDDC apply's
interior-interface coupling blocks in sliced ELL form (csrc/sell.h),
compiled for the host with g++ here (no GPU): on random CSR patterns with
empty rows, long rows and ragged row counts, every CSR entry appears exactly
once, at its row's lane and in its row order; padding carries source -1 and
column 0; the row map is a permutation of the rows, sorted by decreasing
length inside each window of 256 rows; slice lengths are their longest row
and slice offsets their running sum.  A product through the layout (the
GPU kernel's loop, written here in NumPy) equals the CSR product."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WRAPPER = r"""
#include "sell.h"
#include <cstring>
static cbddc::SellHost g_last;
extern "C" long long sell_build(const int* ptr, int nrows, const int* col, const int* src) {
  std::vector<int> p(ptr, ptr + nrows + 1);
  std::vector<int> c(col, col + p[nrows]), s(src, src + p[nrows]);
  g_last = cbddc::build_sell(p, c, s);
  return g_last.steps;
}
extern "C" int sell_slices() { return (int)g_last.len.size(); }
extern "C" void sell_copy(int* off, int* len, int* row, int* col, int* src) {
  std::memcpy(off, g_last.off.data(), g_last.off.size() * sizeof(int));
  std::memcpy(len, g_last.len.data(), g_last.len.size() * sizeof(int));
  std::memcpy(row, g_last.row.data(), g_last.row.size() * sizeof(int));
  std::memcpy(col, g_last.col.data(), g_last.col.size() * sizeof(int));
  std::memcpy(src, g_last.src.data(), g_last.src.size() * sizeof(int));
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("sell")
    src = d / "wrap.cpp"
    src.write_text(WRAPPER)
    so = d / "libsell.so"
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2208_06191_gb300", "csrc"), str(src), "-o", str(so)],
                   check=True)
    L = ctypes.CDLL(str(so))
    L.sell_build.restype = ctypes.c_longlong
    return L


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _build(L, ptr, col, src):
    nrows = len(ptr) - 1
    steps = L.sell_build(_i32(ptr).ctypes.data_as(ctypes.c_void_p), nrows,
                         _i32(col).ctypes.data_as(ctypes.c_void_p), _i32(src).ctypes.data_as(ctypes.c_void_p))
    nsl = L.sell_slices()
    off = np.zeros(nsl + 1, np.int32)
    ln = np.zeros(nsl, np.int32)
    row = np.zeros(nsl * 32, np.int32)
    c = np.zeros(max(steps, 1) * 32, np.int32)
    s = np.zeros(max(steps, 1) * 32, np.int32)
    L.sell_copy(*[a.ctypes.data_as(ctypes.c_void_p) for a in (off, ln, row, c, s)])
    return steps, off, ln, row, c[:steps * 32], s[:steps * 32]


def _random_csr(rng, nrows, ncols, max_len):
    lens = rng.integers(0, max_len + 1, nrows)
    lens[rng.random(nrows) < 0.2] = 0          # empty rows
    if nrows > 3:
        lens[rng.integers(0, nrows)] = 3 * max_len  # one long row
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = rng.integers(0, ncols, ptr[-1]).astype(np.int32)
    src = rng.permutation(ptr[-1]).astype(np.int32)
    return ptr, col, src


@pytest.mark.parametrize("nrows,max_len,seed", [(1, 5, 0), (31, 7, 1), (32, 4, 2), (33, 12, 3),
                                                (257, 9, 4), (1000, 30, 5), (0, 3, 6)])
def test_sliced_layout(lib, nrows, max_len, seed):
    rng = np.random.default_rng(seed)
    ncols = 50
    ptr, col, src = _random_csr(rng, nrows, ncols, max_len)
    steps, off, ln, row, c, s = _build(lib, ptr, col, src)
    nsl = (nrows + 31) // 32
    assert len(ln) == nsl
    lens = np.diff(ptr)
    # row map: a permutation, -1 padding only at the end
    valid = row[row >= 0]
    assert sorted(valid.tolist()) == list(range(nrows))
    assert np.all(row[nrows:] == -1)
    # sorted by decreasing length inside windows of 256 rows (stable)
    for w0 in range(0, nrows, 256):
        win = row[w0:min(nrows, w0 + 256)]
        assert sorted(win.tolist()) == list(range(w0, min(nrows, w0 + 256)))
        wl = lens[win]
        assert np.all(wl[:-1] >= wl[1:])
    # slice lengths and offsets
    for q in range(nsl):
        rows_q = row[32 * q:32 * q + 32]
        assert ln[q] == max([lens[r] for r in rows_q if r >= 0] + [0])
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(ln)]))
    assert steps == off[-1]
    # every entry once, in its row's lane and order; padding -1 / column 0
    seen = np.zeros(ptr[-1], bool)
    for q in range(nsl):
        for lane in range(32):
            r = row[32 * q + lane]
            for k in range(ln[q]):
                p = (off[q] + k) * 32 + lane
                if r >= 0 and k < lens[r]:
                    e = ptr[r] + k
                    assert s[p] == src[e] and c[p] == col[e]
                    assert not seen[e]
                    seen[e] = True
                else:
                    assert s[p] == -1 and c[p] == 0
    assert seen.all()
    # a product through the layout equals the CSR product
    vals = rng.standard_normal(max(ptr[-1], 1))
    x = rng.standard_normal(ncols)
    y_csr = np.array([np.dot(vals[src[ptr[r]:ptr[r + 1]]], x[col[ptr[r]:ptr[r + 1]]])
                      for r in range(nrows)])
    y = np.zeros(nrows)
    for q in range(nsl):
        acc = np.zeros(32)
        for k in range(ln[q]):
            p = (off[q] + k) * 32 + np.arange(32)
            v = np.where(s[p] >= 0, vals[np.maximum(s[p], 0)], 0.0)
            acc += v * x[c[p]]
        for lane in range(32):
            if row[32 * q + lane] >= 0:
                y[row[32 * q + lane]] = acc[lane]
    assert np.allclose(y, y_csr, rtol=1e-13, atol=1e-13)
