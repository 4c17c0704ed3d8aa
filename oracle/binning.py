"""Bubble tracking and binning (Algorithm 1 step 2), brute force (test infrastructure only).

Algorithm 1 step 2 locates each bubble in the lattice and selects the nodes it
interacts with.  Here that is written out from its definition:

* the containing cell of a bubble at x_b is floor(x_b) per axis (cell i spans
  [i, i+1] and holds node i + 1/2), as a linear id (k ny + j) nx + i;
* the nodes a bubble interacts with are the cells whose interval overlaps the
  open window (x_b - n, x_b + n) on every axis, n = width_factor d_b
  (wrapped on a periodic axis, cut at the box on a wall axis);
* for a partition of the box into tiles of shape (tx, ty, tz), a bubble
  belongs to every tile that holds at least one of those cells.  Each tile's
  list is sorted by bubble index.

All arithmetic is float64 and matches the definition exactly (floor / ceil of
x_b -+ n), so the results are integers to compare bit for bit.
"""
import math


def containing_cell(xb, dims):
    """Linear id of the cell holding x_b (clamped to the box)."""
    idx = []
    for a in range(3):
        i = int(math.floor(xb[a]))
        idx.append(min(max(i, 0), dims[a] - 1))
    return (idx[2] * dims[1] + idx[1]) * dims[0] + idx[0]


def support_cells(xb_a, n, length, periodic):
    """Cells of one axis whose interval overlaps (x_b - n, x_b + n), in order."""
    lo = int(math.floor(xb_a - n))
    hi = int(math.ceil(xb_a + n)) - 1
    cells = []
    for i in range(lo, hi + 1):
        if periodic:
            cells.append(i % length)
        elif 0 <= i < length:
            cells.append(i)
    return cells


def tile_lists(xb_list, n_list, active, dims, walls, tile):
    """Per-tile sorted bubble lists.  Returns (offsets[T+1], items[])."""
    nt = [-(-dims[a] // tile[a]) for a in range(3)]
    ntiles = nt[0] * nt[1] * nt[2]
    lists = [[] for _ in range(ntiles)]
    for b, (xb, n) in enumerate(zip(xb_list, n_list)):
        if not active[b]:
            continue
        tiles_axis = []
        for a in range(3):
            periodic = not bool(walls & (1 << (2 * a)))
            cells = support_cells(xb[a], n, dims[a], periodic)
            tiles_axis.append(sorted(set(c // tile[a] for c in cells)))
        for tz in tiles_axis[2]:
            for ty in tiles_axis[1]:
                for tx in tiles_axis[0]:
                    lists[(tz * nt[1] + ty) * nt[0] + tx].append(b)
    offsets = [0]
    items = []
    for lst in lists:
        items.extend(sorted(lst))
        offsets.append(len(items))
    return offsets, items
