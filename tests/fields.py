"""Per-field views of the library's concatenated patch arrays, for parity
norms taken one conserved field at a time (rho, m_x, m_y, m_z, E, b_x, b_y,
b_z), as the FP64 tolerance is stated per field."""
import numpy as np

NAMES = ("rho", "m_x", "m_y", "m_z", "E", "b_x", "b_y", "b_z")


def split_fields(arrays, cells):
    """arrays = (U, bx, by, bz) concatenated over patches; cells[P] = the
    number of cells of patch P.  Returns the eight fields, each concatenated
    over patches."""
    U = np.asarray(arrays[0])
    cells = np.asarray(cells, np.int64)
    offs = np.concatenate([[0], np.cumsum(5 * cells)])
    parts = [[] for _ in range(5)]
    for P, c in enumerate(cells):
        u = U[offs[P]:offs[P + 1]].reshape(5, c)
        for k in range(5):
            parts[k].append(u[k])
    return [np.concatenate(p) for p in parts] + [np.asarray(a) for a in arrays[1:]]


def field_errors(out, ref, cells):
    """Relative L-infinity of each field: max|a - b| / max(max|b|, 1e-300)."""
    a, b = split_fields(out, cells), split_fields(ref, cells)
    return {n: float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), 1e-300)) for n, x, y in zip(NAMES, a, b)}
