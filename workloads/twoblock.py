"""Seeded two-block geometries: two curvilinear blocks that share one face node for node.

Block "-" spans q in [0, 1] from the plane x = 0 to the interface, block "+" from the interface
to x = L1 + L2.  Both map (r, s) to the same (y, z) and place the interface at
x = L1 + d sin(pi r) sin(pi s) (a curved interface when d != 0), so that their q = 1 and q = 0
faces hold the same nodes in the same order.  Each block adds an interior warp that vanishes on
its faces.  Closed-form generators only (numpy or torch)."""
import math


def two_block_maps(L1, L2, Ly, Lz, d=0.0, warp=0.0):
    """(map_minus, map_plus): functions (q, r, s) -> (x, y, z) of the reference coordinates in
    [0, 1]^3 (arrays broadcasting against each other)."""
    def face(r, s, xp):
        return L1 + d * xp.sin(math.pi * r) * xp.sin(math.pi * s)

    def bump(q, r, s, xp):
        # 4 q (1 - q): exactly zero on both q faces, so that the shared face's nodes agree bit for bit
        return warp * 4 * q * (1 - q) * xp.sin(math.pi * r) * xp.sin(math.pi * s)

    def yz(q, r, s, xp):
        b = bump(q, r, s, xp)
        return Ly * r + 0.3 * b * Ly, -Lz + Lz * s + 0.2 * b * Lz

    def xp_of(*a):
        import numpy as np
        for v in a:
            if hasattr(v, "device") and not isinstance(v, np.ndarray):
                import torch
                return torch
        return np

    def minus(q, r, s):
        xp = xp_of(q, r, s)
        b = bump(q, r, s, xp)
        x = q * face(r, s, xp) + 0.1 * b * L1
        y, z = yz(q, r, s, xp)
        return x, y, z

    def plus(q, r, s):
        xp = xp_of(q, r, s)
        b = bump(q, r, s, xp)
        f = face(r, s, xp)
        x = f + q * (L1 + L2 - f) + 0.1 * b * L2
        y, z = yz(q, r, s, xp)
        return x, y, z

    return minus, plus


def block_coordinates(fmap, nodes):
    """Node coordinates [s][r][q] of a map on nq x nr x ns nodes (numpy)."""
    import numpy as np
    nq, nr, ns = nodes
    q = (np.arange(nq) / (nq - 1))[None, None, :]
    r = (np.arange(nr) / (nr - 1))[None, :, None]
    s = (np.arange(ns) / (ns - 1))[:, None, None]
    return [np.broadcast_to(c, (ns, nr, nq)).copy() for c in fmap(q, r, s)]
