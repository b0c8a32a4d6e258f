// Sliced ELL layout of a block-sparse matrix, for the BDDC apply's
// interior-interface coupling blocks.  Host code only.
#pragma once
#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <vector>

namespace cbddc {

// Slice q holds rows row[32 q .. 32 q + 31] (-1 past the last row) and
// len[q] steps starting at step off[q]; step k of lane l is entry k of that
// lane's row: column col[(off[q] + k) 32 + l] and source src[...] (the
// index of the entry in the CSR input; padding past the row's end has
// column 0 and source -1).  Rows are sorted by decreasing length inside
// windows of 8 slices (256 rows, stable), so that a slice's rows have
// similar lengths while neighbouring rows stay together.
struct SellHost {
  std::vector<int> off, len, row, col, src;
  int64_t steps = 0;
};

// ptr: CSR row pointers (rows + 1), col / src: per entry.  Throws
// std::length_error when the layout would need 2^31 steps or more.
inline SellHost build_sell(const std::vector<int>& ptr, const std::vector<int>& col,
                           const std::vector<int>& src) {
  const int nrows = (int)ptr.size() - 1;
  std::vector<int> order(std::max(nrows, 0));
  for (int i = 0; i < nrows; ++i) order[i] = i;
  for (int w0 = 0; w0 < nrows; w0 += 256) {
    const int w1 = std::min(nrows, w0 + 256);
    std::stable_sort(order.begin() + w0, order.begin() + w1,
                     [&](int a, int b) { return ptr[a + 1] - ptr[a] > ptr[b + 1] - ptr[b]; });
  }
  const int nsl = (std::max(nrows, 0) + 31) / 32;
  SellHost S;
  S.off.assign(nsl + 1, 0);
  S.len.assign(nsl, 0);
  S.row.assign((size_t)nsl * 32, -1);
  int64_t steps = 0;
  for (int q = 0; q < nsl; ++q) {
    int L = 0;
    for (int l = 0; l < 32 && 32 * q + l < nrows; ++l) {
      const int r = order[32 * q + l];
      S.row[32 * q + l] = r;
      L = std::max(L, ptr[r + 1] - ptr[r]);
    }
    S.off[q] = (int)steps;
    S.len[q] = L;
    steps += L;
    if (steps >= INT32_MAX) throw std::length_error("sliced coupling layout too large");
  }
  S.off[nsl] = (int)steps;
  S.steps = steps;
  S.col.assign((size_t)steps * 32, 0);
  S.src.assign((size_t)steps * 32, -1);
  for (int q = 0; q < nsl; ++q)
    for (int l = 0; l < 32; ++l) {
      const int r = S.row[32 * q + l];
      if (r < 0) continue;
      for (int k = 0; k < ptr[r + 1] - ptr[r]; ++k) {
        const size_t p = ((size_t)S.off[q] + k) * 32 + l;
        S.col[p] = col[ptr[r] + k];
        S.src[p] = src[ptr[r] + k];
      }
    }
  return S;
}

}  // namespace cbddc
