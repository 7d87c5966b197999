"""Composite ("topological") Vanka patches for Taylor-Hood (P_k, P_{k-1}) on triangles (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3.1 builds one patch per topological entity (vertex, edge, cell) that carries pressure DoFs of
P_{k-1}: the patch holds *all* pressure DoFs on that entity and the velocity DoFs on the closure of
the entity's star.  The star of a vertex is the vertex with its incident edges and cells; the star of
an edge is the edge with its (one or two) incident cells; the star of a cell is the cell.  The closure
of a star is therefore the union of the closed cells in it, so the velocity DoFs of a patch are all
P_k DoFs of every cell that contains the entity.

  k = 2: vertex patches (1 pressure DoF each);
  k = 3: vertex patches + edge patches (1 edge pressure DoF each);
  k = 4: vertex + edge (2 pressure DoFs each) + cell patches (1 pressure DoF each).

Readings where the paper is silent:
* Dirichlet velocity DoFs are left out of every patch (their rows are identity, their columns zero);
* inside a patch DoFs are sorted by global index; patches are ordered vertices (id order), then edges
  (horizontal, vertical, diagonal; each j outer, i inner), then cells (lower, then upper triangles).

This module finds the entity of each P_{k-1} node from its barycentric multi-index in each cell, and
the cells of a star by testing which cells contain the entity -- a generic topological construction.
"""
import numpy as np

from . import exact


def _entity_of_pnode(cell, alpha):
    """The entity (frozenset of vertex coordinates) that owns a P_{k-1} node with barycentric
    multi-index alpha in this cell: the vertices whose barycentric weight is nonzero."""
    return frozenset(v for v, a in zip(cell, alpha) if a > 0)


def entity_order_key(ent, N):
    """Position of an entity in the canonical patch order."""
    vs = sorted(ent, key=lambda v: (v[1], v[0]))
    if len(vs) == 1:
        (i, j), = vs
        return (0, 0, j, i)
    if len(vs) == 2:
        (xa, ya), (xb, yb) = vs
        if ya == yb:                      # horizontal edge (i,j)-(i+1,j)
            return (1, 0, ya, min(xa, xb))
        if xa == xb:                      # vertical edge (i,j)-(i,j+1)
            return (1, 1, min(ya, yb), xa)
        # diagonal (i+1, j)-(i, j+1): lower endpoint first after the sort
        return (1, 2, ya, xb)
    # cell: lower triangle (i,j),(i+1,j),(i,j+1) or upper (i+1,j),(i+1,j+1),(i,j+1)
    xs = sorted(v[0] for v in vs)
    ys = sorted(v[1] for v in vs)
    i, j = xs[0], ys[0]
    upper = (i + 1, j + 1) in ent
    return (2, int(upper), j, i)


def build_patches(space):
    """List of patches; each is (kind, entity, dofs) with dofs a sorted int64 array.

    kind is 'vertex', 'edge' or 'cell'."""
    k = space.k
    mask = space.dirichlet_mask()
    ref_p = exact.lattice_nodes(k - 1)
    # alpha = (k-1-s-t, s, t) are the barycentric weights of (v0, v1, v2)
    pressure_of = {}
    for cell in space.mesh.cells:
        pdofs = space.cell_pdofs(cell)
        for (s, t), g in zip(ref_p, pdofs):
            alpha = (k - 1 - s - t, s, t)
            ent = _entity_of_pnode(cell, alpha)
            pressure_of.setdefault(ent, set()).add(g)
    # cells containing an entity: the cells through one of its vertices that contain all of them
    by_vertex = {}
    for ci, cell in enumerate(space.mesh.cells):
        for v in cell:
            by_vertex.setdefault(v, []).append(ci)
    patches = []
    for ent, pset in pressure_of.items():
        v0 = next(iter(ent))
        cand = by_vertex[v0]
        cells = [space.mesh.cells[ci] for ci in cand if ent <= set(space.mesh.cells[ci])]
        vel = set()
        for cell in cells:
            vel.update(space.cell_vdofs(cell))
        vel = [d for d in vel if not mask[d]]
        dofs = np.array(sorted(vel) + sorted(pset), dtype=np.int64)
        kind = {1: "vertex", 2: "edge", 3: "cell"}[len(ent)]
        patches.append((kind, ent, dofs))
    patches.sort(key=lambda p: entity_order_key(p[1], space.N))
    return patches


def interior_patch_size(k, kind):
    """Closed-form size of an interior patch (no Dirichlet DoF removed).

    vertex: the star has 7 vertices, 12 edges and 6 cells; edge: 4 vertices, 5 edges, 2 cells;
    cell: 3 vertices, 3 edges, 1 cell.  P_k has k-1 nodes inside an edge and (k-1)(k-2)/2 inside a
    cell; P_{k-1} has k-2 per edge and (k-2)(k-3)/2 per cell."""
    e_in = k - 1
    c_in = (k - 1) * (k - 2) // 2
    if kind == "vertex":
        return 2 * (7 + 12 * e_in + 6 * c_in) + 1
    if kind == "edge":
        return 2 * (4 + 5 * e_in + 2 * c_in) + (k - 2)
    if kind == "cell":
        return 2 * (3 + 3 * e_in + c_in) + (k - 2) * (k - 3) // 2
    raise ValueError(kind)
