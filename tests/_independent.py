"""Independent restatements used only to pin the oracle (tests only).

These follow the definitions rather than the oracle's code path:

* ``bfs_labels``: clusters by breadth-first search over open bonds between
  interior nodes, label = smallest member index (Sec. II network; the label
  convention is the project's).
* ``dense_solve``: Kirchhoff's laws written with the bond-node incidence
  matrix B: currents I = W B P, conservation B^T I = 0 at interior nodes, i.e.
  L = B^T W B partitioned into unknown / fixed nodes (Eq. 3), solved densely
  with LAPACK; the flow Q (Eq. 4) is summed from the bond currents.
"""
from collections import deque

import numpy as np


def node_coords(dims):
    n = list(dims) + [1] * (3 - len(dims))
    idx = np.arange(int(np.prod(n)))
    return idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1]), n


def bond_list(dims, planes, periodic=()):
    """All bonds as (i, j, g) with j the node one step along e_d; along a
    periodic axis the last layer's bonds reach back to layer 0."""
    n = list(dims) + [1] * (3 - len(dims))
    out = []
    for d in range(len(dims)):
        m = list(n)
        if d not in periodic:
            m[d] -= 1
        g = np.asarray(planes[d], dtype=np.float64).reshape(-1)
        for z in range(m[2]):
            for y in range(m[1]):
                for x in range(m[0]):
                    b = x + m[0] * (y + m[1] * z)
                    c = [x, y, z]
                    i = c[0] + n[0] * (c[1] + n[1] * c[2])
                    c[d] = (c[d] + 1) % n[d]
                    j = c[0] + n[0] * (c[1] + n[1] * c[2])
                    out.append((i, j, float(g[b])))
    return out


def face_kind(dims, flow_axis):
    xs, ys, zs, n = node_coords(dims)
    c = [xs, ys, zs][flow_axis]
    kind = np.zeros(len(xs), np.int64)
    kind[c == 0] = 1
    kind[c == n[flow_axis] - 1] = 2
    return kind


def bfs_labels(dims, planes, flow_axis=0, periodic=()):
    kind = face_kind(dims, flow_axis)
    N = len(kind)
    adj = [[] for _ in range(N)]
    for i, j, g in bond_list(dims, planes, periodic):
        if g > 0:
            adj[i].append(j)
            adj[j].append(i)
    label = np.full(N, -3, np.int64)
    cls = np.zeros(N, np.int64)
    label[kind == 1] = -1
    label[kind == 2] = -2
    cls[kind == 1] = 4
    cls[kind == 2] = 5
    for s in range(N):
        if kind[s] != 0 or label[s] != -3:
            continue
        comp, flags = [s], 0
        label[s] = s
        dq = deque([s])
        while dq:
            u = dq.popleft()
            for v in adj[u]:
                if kind[v] == 1:
                    flags |= 1
                elif kind[v] == 2:
                    flags |= 2
                elif label[v] == -3:
                    label[v] = s
                    comp.append(v)
                    dq.append(v)
        for u in comp:
            cls[u] = flags
    return label, cls


def dense_solve(dims, planes, flow_axis=0, p_in=1.0, p_out=0.0, periodic=()):
    """Returns (P, Q_in, Q_out) by a dense direct solve on the spanning set."""
    kind = face_kind(dims, flow_axis)
    label, cls = bfs_labels(dims, planes, flow_axis, periodic)
    N = len(kind)
    bonds = bond_list(dims, planes, periodic)
    B = np.zeros((len(bonds), N))
    w = np.zeros(len(bonds))
    for k, (i, j, g) in enumerate(bonds):
        B[k, i] = 1.0
        B[k, j] = -1.0
        w[k] = g
    L = B.T @ (w[:, None] * B)
    P = np.zeros(N)
    P[(cls == 4) | (cls == 1)] = p_in
    P[(cls == 5) | (cls == 2)] = p_out
    U = np.where(cls == 3)[0]
    K = np.where(cls != 3)[0]
    if len(U):
        P[U] = np.linalg.solve(L[np.ix_(U, U)], -L[np.ix_(U, K)] @ P[K])
    current = w * (B @ P)  # current on bond k flows from i to j
    qin = qout = 0.0
    for k, (i, j, g) in enumerate(bonds):
        if kind[i] == 1 and kind[j] == 0:
            qin += current[k]
        if kind[j] == 1 and kind[i] == 0:
            qin -= current[k]
        if kind[i] == 0 and kind[j] == 2:
            qout += current[k]
        if kind[j] == 0 and kind[i] == 2:
            qout -= current[k]
    return P, qin, qout


def read_golden(path):
    vals = {"gx": [], "gy": [], "gz": [], "P": []}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key in vals:
                vals[key].append([float(v) for v in rest])
            else:
                vals[key] = [float(v) for v in rest]
    dims = tuple(int(v) for v in vals["dims"])
    planes = [np.array(vals[k]) for k in ("gx", "gy", "gz")[: len(dims)]]
    return dims, planes, vals


def contracted_graph(dims, planes, flow_axis=0, periodic=()):
    """Adjacency sets of the open-bond graph with every inlet-face node taken
    as the one vertex 'A' and every outlet-face node as 'B' (bonds inside a
    face dropped)."""
    kind = face_kind(dims, flow_axis)
    name = {1: "A", 2: "B"}
    adj = {}
    for i, j, g in bond_list(dims, planes, periodic):
        if not g > 0:
            continue
        u = name.get(int(kind[i]), i)
        v = name.get(int(kind[j]), j)
        if u == v or (isinstance(u, str) and isinstance(v, str)):
            continue
        adj.setdefault(u, set()).add(v)
        adj.setdefault(v, set()).add(u)
    return adj


def simple_path_nodes(dims, planes, flow_axis=0, periodic=(), limit=2_000_000):
    """Brute force over every path from 'A' to 'B' that visits no vertex twice
    (tiny networks only): the set of interior nodes lying on at least one.
    Bonds on such paths are the ones that carry current for generic
    conductances."""
    adj = contracted_graph(dims, planes, flow_axis, periodic)
    on = set()
    if "A" not in adj or "B" not in adj:
        return on
    count = 0
    path = ["A"]
    seen = {"A"}
    stack = [iter(sorted(adj["A"], key=str))]
    while stack:
        nxt = next(stack[-1], None)
        if nxt is None:
            stack.pop()
            seen.discard(path.pop())
            continue
        if nxt in seen:
            continue
        if nxt == "B":
            on.update(v for v in path if not isinstance(v, str))
            count += 1
            if count > limit:
                raise RuntimeError("too many paths for a brute-force check")
            continue
        path.append(nxt)
        seen.add(nxt)
        stack.append(iter(sorted(adj.get(nxt, ()), key=str)))
    return on
