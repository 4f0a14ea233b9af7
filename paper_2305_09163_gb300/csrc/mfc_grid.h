// Non-uniform grid tables (host side); see mfc_grid.cu for the construction
// and the row layout.
#pragma once
#include <vector>

namespace mfc {

constexpr int kGridRow = 28;   // values per cell row (each stored as an FP32 pair)

// Rows for the cells -1..n of one direction with faces faces[0..n]; ghost
// cells mirror (or, periodic, wrap) the interior widths.  false on a bad grid.
bool grid_tables(const double* faces, int n, bool periodic, std::vector<float>& out);

}  // namespace mfc
