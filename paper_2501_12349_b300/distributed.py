"""Element-partitioned findpts across ranks: the global map Psi_G (Sec.
3.1.4) and the multi-rank Find of Sec. 3.2.

Each rank holds a partition of the mesh (its elements, with their own
resident fp_mesh) and issues Find for its own points.  Setup builds Psi_G, a
Cartesian mesh M_G over the union of every rank's element AABBs with N_G
cells per direction; cell i (lexicographic) is owned by rank i % P under the
local index i // P, and its owner stores the ranks whose element AABBs
overlap it.  Find then runs in four steps:

  1. every rank searches its points in its own partition (local_find);
  2. the points found BORDER or NOT_FOUND go to the owner of their M_G cell
     (first exchange), which looks up the cell's ranks in Psi_G and
     forwards each point to every listed rank but the one that issued it
     (second exchange);
  3. those ranks search the points in their partitions and return the
     INTERIOR and BORDER results to the issuing rank (third exchange);
  4. the issuing rank keeps, per point, an INTERIOR result if there is one,
     else the BORDER result with the smallest distance (its own first-step
     result included).

Two readings where the paper is silent: several ranks returning INTERIOR
for one point (a point on a face between partitions) resolve to the lowest
rank, and equal BORDER distances to the lowest rank.  A point outside M_G is
NOT_FOUND without any exchange.

The exchanges are torch.distributed all_to_all_single calls on the tensors
of the local find's device (NCCL for CUDA tensors, gloo for CPU tensors).
This module moves and merges results; the search itself is local_find, on a
GPU the library's fp_findpts (Mesh.find).  Multi-rank runs are tested as
gloo process groups on the CPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist

FP_INTERIOR, FP_BORDER, FP_NOT_FOUND = 0, 1, 2


def _exchange(rows: torch.Tensor, dest: torch.Tensor, group=None) -> torch.Tensor:
    """Sends row i of rows ([n][k] float64) to rank dest[i]; returns the rows
    this rank received ([m][k]), grouped by source rank in rank order, each
    source's rows in their sending order."""
    P = dist.get_world_size(group)
    k = rows.shape[1]
    order = torch.sort(dest, stable=True).indices
    send = rows[order].contiguous()
    counts = torch.bincount(dest, minlength=P).to(torch.int64)
    recv_counts = torch.empty_like(counts)
    dist.all_to_all_single(recv_counts, counts, group=group)
    rc = recv_counts.tolist()
    out = torch.empty((sum(rc), k), dtype=rows.dtype, device=rows.device)
    dist.all_to_all_single(out, send, rc, counts.tolist(), group=group)
    return out


def _cells(x: torch.Tensor, lo: torch.Tensor, scale: torch.Tensor, n: int) -> torch.Tensor:
    """Per-axis cell coordinate floor((x - lo) * scale), clamped to [0, n-1]."""
    t = (x - lo) * scale
    c = torch.where(t >= n, torch.full_like(t, n - 1), torch.floor(t))
    return c.clamp(0, n - 1).to(torch.int64)


@dataclass
class GlobalMap:
    """Psi_G of Sec. 3.1.4 as held by one rank: the bounds and resolution of
    M_G (the same on every rank) and, for the cells this rank owns (global
    index i with i % P == rank, local index i // P), the sorted lists of
    ranks whose element AABBs overlap the cell, in CSR form."""
    d: int
    n: int
    lo: torch.Tensor
    hi: torch.Tensor
    scale: torch.Tensor
    start: torch.Tensor  # [n_local_cells + 1]
    ranks: torch.Tensor  # [nnz]
    world: int
    rank: int

    @staticmethod
    def build(aabb: torch.Tensor, d: int, n_grid: int = 0, group=None) -> "GlobalMap":
        """aabb: this rank's expanded element AABBs [NE_local][2d] (fp_get_boxes
        or Mesh.boxes).  n_grid 0: the smallest n with n^d >= the total
        element count, as for Psi_L.  Collective over the group."""
        P, me = dist.get_world_size(group), dist.get_rank(group)
        dev, f64 = aabb.device, torch.float64
        aabb = aabb.to(f64)
        ne = aabb.shape[0]
        lo = aabb[:, :d].min(0).values if ne else torch.full((d,), float("inf"), dtype=f64, device=dev)
        hi = aabb[:, d:].max(0).values if ne else torch.full((d,), -float("inf"), dtype=f64, device=dev)
        dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
        dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
        total = torch.tensor([ne], dtype=torch.int64, device=dev)
        dist.all_reduce(total, group=group)
        n = n_grid
        if n <= 0:
            n = 1
            while n ** d < int(total.item()):
                n += 1
        ext = hi - lo
        scale = torch.where(ext > 0, n / torch.where(ext > 0, ext, torch.ones_like(ext)), torch.zeros_like(ext))
        # every cell each local element's AABB overlaps
        c0 = _cells(aabb[:, :d], lo, scale, n)
        c1 = _cells(aabb[:, d:], lo, scale, n)
        span = c1 - c0 + 1  # [ne][d]
        cnt = span.prod(1)
        owner_elem = torch.repeat_interleave(torch.arange(ne, device=dev), cnt)
        off = torch.arange(int(cnt.sum().item()), device=dev) - torch.repeat_interleave(torch.cumsum(cnt, 0) - cnt, cnt)
        gid = torch.zeros_like(off)
        mul, rem = 1, off
        for c in range(d):
            s = span[owner_elem, c]
            gid = gid + (c0[owner_elem, c] + rem % s) * mul
            rem = rem // s
            mul *= n
        cells = torch.unique(gid)
        rows = torch.stack([(cells // P).to(f64), torch.full_like(cells, me).to(f64)], 1)
        recv = _exchange(rows, cells % P, group)
        local_cells = (n ** d + P - 1 - me) // P  # global cells i with i % P == me
        key = recv[:, 0].to(torch.int64) * P + recv[:, 1].to(torch.int64)
        key = torch.unique(key)  # sorted: by local cell, then rank; duplicates removed
        lc, rk = key // P, key % P
        start = torch.zeros(local_cells + 1, dtype=torch.int64, device=dev)
        start[1:] = torch.cumsum(torch.bincount(lc, minlength=local_cells), 0)
        return GlobalMap(d, n, lo, hi, scale, start, rk, P, me)

    def cell_of(self, x: torch.Tensor) -> torch.Tensor:
        """Global M_G cell of each point, -1 outside M_G or non-finite."""
        inside = torch.all((x >= self.lo) & (x <= self.hi), dim=1)
        c = _cells(torch.where(torch.isfinite(x), x, torch.zeros_like(x)), self.lo, self.scale, self.n)
        gid = torch.zeros(x.shape[0], dtype=torch.int64, device=x.device)
        mul = 1
        for k in range(self.d):
            gid = gid + c[:, k] * mul
            mul *= self.n
        return torch.where(inside, gid, torch.full_like(gid, -1))

    def ranks_of(self, local_cell: torch.Tensor):
        """(flat rank list, row index into local_cell) of owned cells."""
        a, b = self.start[local_cell], self.start[local_cell + 1]
        cnt = b - a
        row = torch.repeat_interleave(torch.arange(local_cell.shape[0], device=local_cell.device), cnt)
        pos = torch.arange(int(cnt.sum().item()), device=local_cell.device) - torch.repeat_interleave(
            torch.cumsum(cnt, 0) - cnt, cnt)
        return self.ranks[a[row] + pos], row


def find(local_find, pts: torch.Tensor, gmap: GlobalMap, group=None):
    """Multi-rank Find of Sec. 3.2 (collective over the group).

    local_find(pts [n][d] float64) -> (code int32 [n], elem int32 [n],
    r float64 [n][dr], dist2 float64 [n]) searches this rank's partition.
    Returns (code, rank, elem, r, dist2) for this rank's points: rank is the
    rank whose element elem (its local index there) holds the result, -1
    where NOT_FOUND."""
    P, me = gmap.world, gmap.rank
    dev, f64 = pts.device, torch.float64
    d = gmap.d
    n = pts.shape[0]
    code, elem, r, dist2 = local_find(pts)
    code, elem, r, dist2 = code.to(torch.int64), elem.to(torch.int64), r.to(f64), dist2.to(f64)
    dr = r.shape[1]
    rank = torch.where(code != FP_NOT_FOUND, torch.full_like(code, me), torch.full_like(code, -1))

    # 1st exchange: points not INTERIOR here, to the owners of their M_G cells
    idx = torch.nonzero(code != FP_INTERIOR).flatten()
    cell = gmap.cell_of(pts[idx])
    keep = cell >= 0
    idx, cell = idx[keep], cell[keep]
    rows = torch.cat([torch.full((idx.shape[0], 1), float(me), dtype=f64, device=dev),
                      idx[:, None].to(f64), (cell // P)[:, None].to(f64), pts[idx].to(f64)], 1)
    recv = _exchange(rows, cell % P, group)

    # 2nd exchange: the owner forwards each point to the cell's other ranks
    origin = recv[:, 0].to(torch.int64)
    to, row = gmap.ranks_of(recv[:, 2].to(torch.int64))
    fwd = to != origin[row]
    to, row = to[fwd], row[fwd]
    rows2 = torch.cat([recv[row][:, :2], recv[row][:, 3:]], 1)
    recv2 = _exchange(rows2, to, group)

    # 3rd exchange: search here, return INTERIOR / BORDER results to the issuer
    if recv2.shape[0]:
        c2, e2, r2, d2 = local_find(recv2[:, 2:].contiguous())
        c2, e2 = c2.to(torch.int64), e2.to(torch.int64)
    else:
        c2 = torch.empty(0, dtype=torch.int64, device=dev)
        e2 = torch.empty(0, dtype=torch.int64, device=dev)
        r2 = torch.empty((0, dr), dtype=f64, device=dev)
        d2 = torch.empty(0, dtype=f64, device=dev)
    ok = c2 != FP_NOT_FOUND
    rows3 = torch.cat([recv2[ok][:, 1:2], c2[ok][:, None].to(f64), torch.full((int(ok.sum().item()), 1), float(me),
                      dtype=f64, device=dev), e2[ok][:, None].to(f64), r2[ok].to(f64), d2[ok][:, None].to(f64)], 1)
    back = _exchange(rows3, recv2[ok][:, 0].to(torch.int64), group)

    # merge: INTERIOR first (lowest rank), else the smallest BORDER distance
    # (then the lowest rank); this rank's own result takes part
    mine = code != FP_NOT_FOUND
    cand_idx = torch.cat([torch.nonzero(mine).flatten(), back[:, 0].to(torch.int64)])
    cand_code = torch.cat([code[mine], back[:, 1].to(torch.int64)])
    cand_rank = torch.cat([rank[mine], back[:, 2].to(torch.int64)])
    cand_elem = torch.cat([elem[mine], back[:, 3].to(torch.int64)])
    cand_r = torch.cat([r[mine], back[:, 4:4 + dr]])
    cand_d2 = torch.cat([dist2[mine], back[:, 4 + dr]])
    d2key = torch.where(cand_code == FP_INTERIOR, torch.zeros_like(cand_d2), cand_d2)
    order = torch.sort(cand_rank, stable=True).indices
    for key in (d2key, cand_code, cand_idx):
        order = order[torch.sort(key[order], stable=True).indices]
    first = torch.ones(order.shape[0], dtype=torch.bool, device=dev)
    s_idx = cand_idx[order]
    first[1:] = s_idx[1:] != s_idx[:-1]
    sel = order[first]
    out_code = torch.full((n,), FP_NOT_FOUND, dtype=torch.int64, device=dev)
    out_rank = torch.full((n,), -1, dtype=torch.int64, device=dev)
    out_elem = torch.full((n,), -1, dtype=torch.int64, device=dev)
    out_r = torch.zeros((n, dr), dtype=f64, device=dev)
    out_d2 = torch.full((n,), float("inf"), dtype=f64, device=dev)
    p = cand_idx[sel]
    out_code[p], out_rank[p], out_elem[p] = cand_code[sel], cand_rank[sel], cand_elem[sel]
    out_r[p], out_d2[p] = cand_r[sel], cand_d2[sel]
    return out_code.to(torch.int32), out_rank.to(torch.int32), out_elem.to(torch.int32), out_r, out_d2
