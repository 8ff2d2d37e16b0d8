"""Network and tree containers and their on-disk formats.

Network (Eq. 1 of the paper: a set of tensors placed on graph vertices, each
bond an index shared by exactly two tensors; no open indices, so the
contraction is a scalar Z):

    binary, little-endian
    8 bytes   magic b"TNNET1\\0\\0"
    int64     n_bonds, n_tensors
    int64     bond_dims[n_bonds]
    per tensor: int64 ndim, int64 bond_ids[ndim]
    per tensor: float64 data, row-major over that tensor's listed bond order

Ordered approximate contraction tree (Fig. 2B/C: a sequence of pairwise
contractions and bond compressions), text:

    tntree 1
    inputs <N>
    C i j k      contract live tensors i and j into the new id k
    S i j        compress all bonds shared by i and j (runs iff their
                 product exceeds chi)

Ids 0..N-1 are the network's tensors; each C creates the next id N, N+1, ...
"""
from __future__ import annotations

import dataclasses
import struct
from typing import List, Sequence, Tuple

import numpy as np

MAGIC = b"TNNET1\0\0"


@dataclasses.dataclass
class Network:
    """Tensors with bond lists; ``bond_dims[b]`` is the size of bond ``b``."""

    bond_dims: List[int]
    bonds: List[List[int]]           # per tensor: bond ids in storage order
    data: List[np.ndarray]           # per tensor: float64 array, shape = dims of its bonds

    @property
    def n_tensors(self) -> int:
        return len(self.bonds)

    def shape(self, t: int) -> Tuple[int, ...]:
        return tuple(self.bond_dims[b] for b in self.bonds[t])

    def validate(self) -> None:
        count = [0] * len(self.bond_dims)
        for t, bl in enumerate(self.bonds):
            if len(set(bl)) != len(bl):
                raise ValueError(f"tensor {t} lists a bond twice")
            for b in bl:
                if not 0 <= b < len(self.bond_dims):
                    raise ValueError(f"tensor {t}: bond id {b} out of range")
                count[b] += 1
            if tuple(self.data[t].shape) != self.shape(t):
                raise ValueError(f"tensor {t}: data shape {self.data[t].shape} != {self.shape(t)}")
        for b, c in enumerate(count):
            if c != 2:
                raise ValueError(f"bond {b} appears {c} times (must be exactly 2)")

    def copy(self) -> "Network":
        return Network(list(self.bond_dims), [list(b) for b in self.bonds],
                       [np.array(d, dtype=np.float64, copy=True) for d in self.data])


@dataclasses.dataclass
class Tree:
    """Ordered approximate contraction tree: ops ('C', i, j, k) or ('S', i, j)."""

    n_inputs: int
    ops: List[tuple]

    def as_int_array(self) -> np.ndarray:
        """(n_ops, 4) int32 rows: kind (0 = C, 1 = S), i, j, k (-1 for S)."""
        out = np.full((len(self.ops), 4), -1, dtype=np.int32)
        for r, op in enumerate(self.ops):
            if op[0] == "C":
                out[r] = (0, op[1], op[2], op[3])
            else:
                out[r] = (1, op[1], op[2], -1)
        return out

    def n_contractions(self) -> int:
        return sum(1 for op in self.ops if op[0] == "C")


def write_network(path: str, net: Network) -> None:
    net.validate()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<qq", len(net.bond_dims), net.n_tensors))
        f.write(np.asarray(net.bond_dims, dtype="<i8").tobytes())
        for bl in net.bonds:
            f.write(struct.pack("<q", len(bl)))
            f.write(np.asarray(bl, dtype="<i8").tobytes())
        for d in net.data:
            f.write(np.ascontiguousarray(d, dtype="<f8").tobytes())


def read_network(path: str) -> Network:
    with open(path, "rb") as f:
        buf = f.read()
    if buf[:8] != MAGIC:
        raise ValueError("not a TNNET1 file")
    off = 8
    nb, nt = struct.unpack_from("<qq", buf, off)
    off += 16
    dims = np.frombuffer(buf, dtype="<i8", count=nb, offset=off).tolist()
    off += 8 * nb
    bonds = []
    for _ in range(nt):
        (nd,) = struct.unpack_from("<q", buf, off)
        off += 8
        bonds.append(np.frombuffer(buf, dtype="<i8", count=nd, offset=off).tolist())
        off += 8 * nd
    data = []
    for bl in bonds:
        shp = tuple(dims[b] for b in bl)
        cnt = int(np.prod(shp, dtype=np.int64))
        data.append(np.frombuffer(buf, dtype="<f8", count=cnt, offset=off).reshape(shp).copy())
        off += 8 * cnt
    net = Network(dims, bonds, data)
    net.validate()
    return net


def write_tree(path: str, tree: Tree) -> None:
    with open(path, "w") as f:
        f.write("tntree 1\n")
        f.write(f"inputs {tree.n_inputs}\n")
        for op in tree.ops:
            f.write(" ".join(str(x) for x in op) + "\n")


def read_tree(path: str) -> Tree:
    ops: list = []
    n_inputs = None
    with open(path) as f:
        for ln, line in enumerate(f):
            s = line.split("#", 1)[0].strip()
            if not s:
                continue
            tok = s.split()
            if tok[0] == "tntree":
                continue
            if tok[0] == "inputs":
                n_inputs = int(tok[1])
            elif tok[0] == "C" and len(tok) == 4:
                ops.append(("C", int(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "S" and len(tok) == 3:
                ops.append(("S", int(tok[1]), int(tok[2])))
            else:
                raise ValueError(f"tree line {ln + 1}: cannot parse {line!r}")
    if n_inputs is None:
        raise ValueError("tree file has no 'inputs' line")
    return Tree(n_inputs, ops)


def edges_to_bonds(n: int, edges: Sequence[Tuple[int, int]]) -> List[List[int]]:
    """Bond list per vertex: bond id = edge index, listed in ascending edge order."""
    bonds: List[List[int]] = [[] for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        if u == v:
            raise ValueError("self-loop edge")
        bonds[u].append(e)
        bonds[v].append(e)
    return bonds
