"""Mesh connectivity and affine geometry for the oracle.

Readings (the paper's grids are 2D; Sec. III-A describes face units E_i and
cell units C_i without fixing conventions):
  * reference element: the unit tetrahedron with vertices (0,0,0), (1,0,0),
    (0,1,0), (0,0,1); x = x_0 + J xi with J = [x_1 - x_0, x_2 - x_0, x_3 - x_0];
  * local face f is the face opposite local vertex f; its vertices are the
    other three local vertices in increasing local order;
  * two faces are the same face when their sorted global vertex-id triples
    agree (periodic images share vertex ids); a face with no partner is a
    boundary face and takes the element's boundary tag for it.
"""
from __future__ import annotations

import numpy as np

REF_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
FACE_VERTS = [[k for k in range(4) if k != f] for f in range(4)]


def jacobians(tet_xyz):
    """J [ne,3,3] (columns x_k - x_0), det J [ne], J^-1 [ne,3,3]."""
    x = np.asarray(tet_xyz, dtype=np.float64)
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    return J, det, Jinv


def match_faces(tet_vid, bc_tag=None):
    """Neighbour element nbr[e,f] (-1 on the boundary), its local face
    nbr_face[e,f] and the boundary type btype[e,f] (0 interior)."""
    vid = np.asarray(tet_vid, dtype=np.int64)
    ne = vid.shape[0]
    keys = np.empty((ne, 4, 3), dtype=np.int64)
    for f in range(4):
        keys[:, f, :] = np.sort(vid[:, FACE_VERTS[f]], axis=1)
    flat = keys.reshape(-1, 3)
    order = np.lexsort((flat[:, 2], flat[:, 1], flat[:, 0]))
    sk = flat[order]
    same_next = np.all(sk[1:] == sk[:-1], axis=1)
    if np.any(same_next[1:] & same_next[:-1]):
        raise ValueError("a face is shared by more than two tetrahedra")
    nbr = -np.ones(ne * 4, dtype=np.int64)
    idx = np.nonzero(same_next)[0]
    a, b = order[idx], order[idx + 1]
    nbr[a] = b
    nbr[b] = a
    nbr_elem = np.where(nbr >= 0, nbr // 4, -1).reshape(ne, 4)
    nbr_face = np.where(nbr >= 0, nbr % 4, -1).reshape(ne, 4)
    btype = np.zeros((ne, 4), dtype=np.int64)
    bnd = nbr_elem < 0
    if np.any(bnd):
        if bc_tag is None:
            raise ValueError("unmatched face without a boundary tag")
        tag = np.asarray(bc_tag, dtype=np.int64)
        if np.any(tag[bnd] == 0):
            raise ValueError("unmatched face tagged interior")
        btype[bnd] = tag[bnd]
    return nbr_elem, nbr_face, btype


def face_normal_area(tet_xyz, e, f):
    """Outward unit normal [n,3] and area [n] of local face f of elements e,
    from the physical vertex coordinates."""
    x = np.asarray(tet_xyz)[e]
    fv = FACE_VERTS[f]
    a, b, c = x[:, fv[0]], x[:, fv[1]], x[:, fv[2]]
    N = np.cross(b - a, c - a)
    out = np.sum(N * (x[:, f] - a), axis=1) > 0.0          # points toward the opposite vertex
    N[out] *= -1.0
    area2 = np.linalg.norm(N, axis=1)
    return N / area2[:, None], 0.5 * area2
