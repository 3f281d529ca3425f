"""The library's MD checkpoint files on the host, without a GPU context:
inspect a stored state, derive a new starting state from it, or write one
from numpy arrays for sxl_checkpoint_read.

Format (the one sxl_checkpoint_write writes, all little-endian):
  8 bytes  magic "SXLCKPT1"
  72 bytes header: uint32 version (1), uint32 header size (72), int32 N_at,
           int32 length of n (n2), int32 kmax, int32 precision, int32
           l_resolved, int32 reserved, int64 step counter, float64 mu,
           float64 previous mu, uint64 payload bytes, uint64 FNV-1a 64-bit
           hash of the payload
  payload  float64: R (N_at x 3), V (N_at x 3), the n history (kmax + 1
           vectors of n2, newest first), F (N_at x 3), Kf (n2), K0 (n2 x n2)
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"SXLCKPT1"
_HEADER = struct.Struct("<IIiiiiiiqddQQ")
_FNV_OFFSET, _FNV_PRIME, _MASK = 14695981039346656037, 1099511628211, (1 << 64) - 1


def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64 bits (the published constants), over the bytes of data."""
    h = _FNV_OFFSET
    for b in data:
        h = ((h ^ b) * _FNV_PRIME) & _MASK
    return h


def _layout(nat: int, n2: int, kmax: int):
    k1 = kmax + 1
    return [("R", (nat, 3)), ("V", (nat, 3)), ("nhist", (k1, n2)), ("F", (nat, 3)),
            ("Kf", (n2,)), ("K0", (n2, n2))]


def read(path, verify: bool = True) -> dict:
    """The checkpoint at path as a dict of header fields and numpy arrays.
    verify: check the payload against its hash (pure Python, about a
    second per 10 MB).  Raises ValueError for another magic, version or
    size, or a payload that does not match its hash."""
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != MAGIC:
        raise ValueError("not a checkpoint: bad magic")
    if len(raw) < 8 + _HEADER.size:
        raise ValueError("truncated header")
    (version, hbytes, nat, n2, kmax, precision, l_resolved, _, md_step, mu, mu_prev,
     pbytes, h) = _HEADER.unpack_from(raw, 8)
    if version != 1 or hbytes != _HEADER.size:
        raise ValueError(f"unsupported checkpoint version {version} / header {hbytes}")
    payload = raw[8 + _HEADER.size:]
    count = sum(int(np.prod(s)) for _, s in _layout(nat, n2, kmax))
    if pbytes != 8 * count or len(payload) != pbytes:
        raise ValueError("payload size does not match the header")
    if verify and fnv1a64(payload) != h:
        raise ValueError("payload does not match its hash")
    arr = np.frombuffer(payload, dtype="<f8")
    out = dict(version=version, n_atoms=nat, n2=n2, kmax=kmax, precision=precision,
               l_resolved=l_resolved, md_step=md_step, mu=mu, mu_prev=mu_prev)
    off = 0
    for name, shape in _layout(nat, n2, kmax):
        size = int(np.prod(shape))
        out[name] = arr[off:off + size].reshape(shape).copy()
        off += size
    return out


def write(path, ck: dict) -> None:
    """Writes ck (the keys read() returns) in the checkpoint format."""
    nat, n2, kmax = int(ck["n_atoms"]), int(ck["n2"]), int(ck["kmax"])
    parts = []
    for name, shape in _layout(nat, n2, kmax):
        a = np.ascontiguousarray(ck[name], dtype="<f8")
        if a.shape != shape:
            raise ValueError(f"{name}: shape {a.shape}, expected {shape}")
        parts.append(a.tobytes())
    payload = b"".join(parts)
    header = _HEADER.pack(1, _HEADER.size, nat, n2, kmax, int(ck.get("precision", 0)),
                          int(ck.get("l_resolved", 0)), 0, int(ck.get("md_step", 0)),
                          float(ck["mu"]), float(ck.get("mu_prev", float("nan"))),
                          len(payload), fnv1a64(payload))
    with open(path, "wb") as f:
        f.write(MAGIC + header + payload)
