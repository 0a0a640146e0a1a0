"""Helpers shared by the GPU parity tests (no method arithmetic)."""
import numpy as np

from oracle import oracle as O


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def slot_dofs(prob, level_n, node):
    """Global DoF of every cached-row slot of the patch of ``node`` (slot order
    of fc_patch_rows), -1 for slots outside the grid."""
    dim = prob.dim
    nd = dim + 1
    nn = [k + 1 for k in level_n]
    idx = [node % nn[0], (node // nn[0]) % nn[1], node // (nn[0] * nn[1]) if dim == 3 else 0]
    out = []
    r5 = 5 if dim == 3 else 1
    for dz in range(r5):
        for dy in range(5):
            for dx in range(5):
                off = (dx - 2, dy - 2, dz - 2 if dim == 3 else 0)
                b = [idx[k] + off[k] for k in range(3)]
                inside = all(0 <= b[k] < nn[k] for k in range(dim))
                nb = b[0] + nn[0] * (b[1] + nn[1] * b[2]) if inside else -1
                for c in range(dim):
                    out.append(nb * nd + c if inside else -1)
    r3 = 3 if dim == 3 else 1
    for dz in range(r3):
        for dy in range(3):
            for dx in range(3):
                off = (dx - 1, dy - 1, dz - 1 if dim == 3 else 0)
                b = [idx[k] + off[k] for k in range(3)]
                inside = all(0 <= b[k] < nn[k] for k in range(dim))
                nb = b[0] + nn[0] * (b[1] + nn[1] * b[2]) if inside else -1
                out.append(nb * nd + dim if inside else -1)
    return np.array(out, dtype=np.int64)


def oracle_rows_in_slots(level: "O.Level", prob, level_n, node):
    """Oracle owned rows of L_i^{-1} scattered into the slot layout."""
    rows, dofs, own = level.patch_inverse_rows(node)
    pos = {int(d): q for q, d in enumerate(dofs)}
    sd = slot_dofs(prob, level_n, node)
    nd = prob.dim + 1
    out = np.zeros((nd, len(sd)))
    for k in range(nd):
        if own[k] < 0:
            continue
        for j, d in enumerate(sd):
            q = pos.get(int(d))
            if q is not None:
                out[k, j] = rows[k, q]
    return out


def oracle_patch_update(level: "O.Level", prob, node, b, x, omega, with_scale=False):
    """omega * (L_i^{-1} R_i r)[owned] for one patch, r = b - L x computed from
    the oracle's own rows of L at the patch DoFs (no assembled operator).
    with_scale: also return, per owned component, omega * sum_j |c_j r_j|
    (the magnitude that rounding of the dot product scales with)."""
    rows, dofs, own = level.patch_inverse_rows(node)
    R, rhs = level.dof_rows(dofs)
    nd = prob.dim + 1
    nn = [k + 1 for k in prob.level_n(prob.nlevels)]
    r = np.zeros(len(dofs))
    for q, d in enumerate(dofs):
        nodeq = d // nd
        iq = [nodeq % nn[0], (nodeq // nn[0]) % nn[1], nodeq // (nn[0] * nn[1]) if prob.dim == 3 else 0]
        s = 0.0
        nnb = 27 if prob.dim == 3 else 9
        for t in range(nnb):
            off = (t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1 if prob.dim == 3 else 0)
            b2 = [iq[k] + off[k] for k in range(3)]
            if not all(0 <= b2[k] < nn[k] for k in range(prob.dim)):
                continue
            nbn = b2[0] + nn[0] * (b2[1] + nn[1] * b2[2])
            for cb in range(nd):
                s += R[q, t, cb] * x[nbn * nd + cb]
        r[q] = b[d] - s
    upd, scale = {}, {}
    for c in range(nd):
        if own[c] >= 0:
            upd[c] = omega * float(rows[c] @ r)
            scale[c] = omega * float(np.abs(rows[c]) @ np.abs(r))
    return (upd, scale) if with_scale else upd
