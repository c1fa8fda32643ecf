"""Latitude-band partition of one analysis over several ranks (host logic).

The sub-domains of Section 3 are independent during the analysis (Algorithm 2):
each needs the background only on its tile plus an r-wide boundary.  A rank
owns a contiguous band of sub-domain rows (tiles of sub_lat latitudes) and
analyses a local grid made of its band plus one whole tile row on each side
(clipped at the poles).  The extra tile rows keep the local tiling aligned with
the global one (the local grid starts on a tile boundary) and hold the r-wide
boundary of the band's tiles (sub_lat >= r); their own analyses are discarded.
So the analysis of every owned tile, and every owned row of T, is the global
one: the predecessors of an owned row and the extended box of an owned tile
lie inside the local grid.

Data movement, through torch.distributed (any backend):
  * forward: one halo scatter -- each rank sends the background rows of its
    band that a neighbour's local grid needs (one tile row on each side), then
    gathers the owned rows of X^a;
  * reverse: the gradient of a loss of X^a comes back from each local problem
    on the whole local grid; the parts on rows a neighbour owns (the boundary
    of the band's tiles reaches into them) are sent to that neighbour and added
    (the reverse of the scatter), and so are the parts for the observations of
    those rows.

Arrays are member-major [N][n] with variable-major labels; a band of latitude
rows is a slice of the [N, planes, nlat, nlon] view (planes = the levels of all
variables).  The compute itself is a callable (the library on a GPU, or any
other implementation of the same analysis).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Band:
    rank: int
    lat0: int   # first owned latitude
    lat1: int   # end of the owned latitudes
    lo: int     # first latitude of the local grid
    hi: int     # end of the local grid


def band_plan(w, world: int):
    """Contiguous bands of sub-domain rows, as even as the rows allow."""
    nrows = -(-w.nlat // w.sub_lat)
    if world < 1 or world > nrows:
        raise ValueError(f"{world} ranks for {nrows} sub-domain rows")
    bands = []
    start = 0
    for k in range(world):
        cnt = nrows // world + (1 if k < nrows % world else 0)
        lat0 = start * w.sub_lat
        lat1 = min(w.nlat, (start + cnt) * w.sub_lat)
        lo = max(0, lat0 - w.sub_lat)
        hi = min(w.nlat, lat1 + w.sub_lat)
        bands.append(Band(k, lat0, lat1, lo, hi))
        start += cnt
    return bands


def planes(w) -> int:
    return w.nvar_3d * w.nlev + w.nvar_2d


def grid_view(X, w):
    """[N][n] -> [N, planes, nlat, nlon] (a view)."""
    return X.reshape(X.shape[0], planes(w), w.nlat, w.nlon)


def local_workload(w, band: Band):
    """The local problem of a band: the same grid on latitudes [lo, hi)."""
    return w.with_(nlat=band.hi - band.lo)


def labels_rows(w, lat_lo: int, lat_hi: int):
    """Global labels of the latitudes [lat_lo, lat_hi), in local label order."""
    lab = np.arange(w.n).reshape(planes(w), w.nlat, w.nlon)
    return lab[:, lat_lo:lat_hi, :].reshape(-1)


def local_observations(w, band: Band, obs_idx):
    """(positions in the global observation list, local labels) of the
    observations whose component lies in the band's local grid."""
    obs_idx = np.asarray(obs_idx, dtype=np.int64)
    glab = labels_rows(w, band.lo, band.hi)
    loc = np.full(w.n, -1, dtype=np.int64)
    loc[glab] = np.arange(glab.size)
    l = loc[obs_idx]
    keep = np.nonzero(l >= 0)[0]
    order = np.argsort(l[keep], kind="stable")      # local labels increasing
    return keep[order], l[keep][order]


def _send_recv(dist, torch, send, dst, recv_shape, src, dtype):
    """Exchange with neighbours (None = no neighbour on that side)."""
    reqs = []
    if send is not None and dst is not None:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send)), dst))
    buf = None
    if src is not None:
        buf = torch.empty(recv_shape, dtype=dtype)
        reqs.append(dist.irecv(buf, src))
    for r in reqs:
        r.wait()
    return None if buf is None else buf.numpy()


def halo_scatter(dist, w, bands, rank, X_owned):
    """Forward exchange: X_owned [N, planes, lat1 - lat0, nlon] (this rank's
    band) -> the local grid's rows [N, planes, hi - lo, nlon], the rows below
    and above the band received from the neighbours."""
    import torch
    b = bands[rank]
    N = X_owned.shape[0]
    out = np.empty((N, planes(w), b.hi - b.lo, w.nlon), dtype=X_owned.dtype)
    out[:, :, b.lat0 - b.lo:b.lat1 - b.lo] = X_owned
    dt = torch.from_numpy(X_owned[:0]).dtype
    # send my lowest tile row down, receive the upper neighbour's lowest
    lower = rank - 1 if rank > 0 else None
    upper = rank + 1 if rank + 1 < len(bands) else None
    for direction in (0, 1):
        if direction == 0:   # to the rank below: my first rows; from the rank above: its first
            dst, src = lower, upper
            send = X_owned[:, :, :bands[lower].hi - b.lat0] if lower is not None else None
            nrecv = b.hi - b.lat1 if upper is not None else 0
        else:                # to the rank above: my last rows; from the rank below: its last
            dst, src = upper, lower
            send = X_owned[:, :, bands[upper].lo - b.lat0:] if upper is not None else None
            nrecv = b.lat0 - b.lo if lower is not None else 0
        got = _send_recv(dist, torch, send, dst, (N, planes(w), nrecv, w.nlon), src, dt)
        if got is not None:
            if direction == 0:
                out[:, :, b.lat1 - b.lo:] = got
            else:
                out[:, :, :b.lat0 - b.lo] = got
    return out


def halo_reduce(dist, w, bands, rank, G_local):
    """Reverse exchange: G_local [N, planes, hi - lo, nlon] (a gradient on the
    local grid) -> this rank's band [N, planes, lat1 - lat0, nlon] with the
    neighbours' contributions to its rows added (the reverse of halo_scatter)."""
    import torch
    b = bands[rank]
    N = G_local.shape[0]
    own = G_local[:, :, b.lat0 - b.lo:b.lat1 - b.lo].copy()
    dt = torch.from_numpy(G_local[:0]).dtype
    lower = rank - 1 if rank > 0 else None
    upper = rank + 1 if rank + 1 < len(bands) else None
    for direction in (0, 1):
        if direction == 0:   # my rows below the band belong to the rank below
            dst, src = lower, upper
            send = G_local[:, :, :b.lat0 - b.lo] if lower is not None else None
            nrecv = bands[upper].lat0 - bands[upper].lo if upper is not None else 0
        else:                # my rows above the band belong to the rank above
            dst, src = upper, lower
            send = G_local[:, :, b.lat1 - b.lo:] if upper is not None else None
            nrecv = bands[lower].hi - bands[lower].lat1 if lower is not None else 0
        got = _send_recv(dist, torch, send, dst, (N, planes(w), nrecv, w.nlon), src, dt)
        if got is not None:
            if direction == 0:   # the upper neighbour's rows below its band: my last rows
                own[:, :, own.shape[2] - nrecv:] += got
            else:                # the lower neighbour's rows above its band: my first rows
                own[:, :, :nrecv] += got
    return own


def obs_reduce(dist, w, bands, rank, obs_idx, local_pos, vals_local):
    """Per-observation gradients of the local problem (indexed like local_pos,
    positions in the global list) summed over the ranks whose local grid holds
    the observation (all-reduce of a full-length vector)."""
    import torch
    full = np.zeros(len(obs_idx), dtype=np.float64)
    full[local_pos] = vals_local
    t = torch.from_numpy(full)
    dist.all_reduce(t)
    return t.numpy()


def gather_owned(dist, w, bands, rank, X_owned_band):
    """All ranks' bands [N, planes, lat1 - lat0, nlon] -> the global [N][n]
    (bands padded to the tallest for the all-gather, then cut)."""
    import torch
    N = X_owned_band.shape[0]
    tallest = max(bb.lat1 - bb.lat0 for bb in bands)
    mine = np.zeros((N, planes(w), tallest, w.nlon))
    mine[:, :, :X_owned_band.shape[2]] = X_owned_band
    if len(bands) == 1:
        parts = [torch.from_numpy(mine)]
    else:
        parts = [torch.empty_like(torch.from_numpy(mine)) for _ in bands]
        dist.all_gather(parts, torch.from_numpy(mine))
    full = np.concatenate([p.numpy()[:, :, :bb.lat1 - bb.lat0] for p, bb in zip(parts, bands)],
                          axis=2)
    return full.reshape(N, -1)
