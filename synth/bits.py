"""Bit-vector packing helpers (layout only, no method arithmetic)."""

import numpy as np


def n_words(n_qubits: int) -> int:
    """Number of 64-bit words per N-bit vector."""
    return max(1, (int(n_qubits) + 63) // 64)


def pack_ints(values, n_qubits: int) -> np.ndarray:
    """Python ints (bit i = qubit i) -> uint64 array [n, W]."""
    W = n_words(n_qubits)
    vals = list(values)
    out = np.zeros((len(vals), W), dtype=np.uint64)
    mask = (1 << 64) - 1
    for r, v in enumerate(vals):
        v = int(v)
        if v < 0 or v >> max(int(n_qubits), 1):
            raise ValueError(f"value {v:#x} does not fit in {n_qubits} qubits")
        for w in range(W):
            out[r, w] = (v >> (64 * w)) & mask
    return out


def unpack_ints(arr: np.ndarray) -> list:
    """uint64 array [n, W] -> list of Python ints."""
    arr = np.asarray(arr, dtype=np.uint64)
    if arr.ndim == 1:
        arr = arr[:, None]
    out = []
    for row in arr:
        v = 0
        for w in range(arr.shape[1] - 1, -1, -1):
            v = (v << 64) | int(row[w])
        out.append(v)
    return out


def from_paper_string(s: str) -> int:
    """Paper notation 'x_0 x_1 ... x_{N-1}' (e.g. '1100') -> int with bit i = x_i."""
    return sum(1 << i for i, ch in enumerate(s) if ch == "1")


def to_paper_string(v: int, n_qubits: int) -> str:
    """Inverse of :func:`from_paper_string`."""
    return "".join("1" if (v >> i) & 1 else "0" for i in range(n_qubits))


def popcount_rows(arr: np.ndarray) -> np.ndarray:
    """Hamming weight of each row of a uint64 [n, W] array."""
    arr = np.asarray(arr, dtype=np.uint64)
    if arr.ndim == 1:
        arr = arr[:, None]
    return np.bitwise_count(arr).sum(axis=1).astype(np.int64)
