"""Sharding of an all-pairs job over ranks (one process per GPU).

Definition 1's result is the disjoint union, over start vertices, of each
start vertex's rows, so the start vertices partition the job: rank r of N
takes every N-th batch of consecutive start vertices and no rows cross
ranks.  The only exchange is the final combination of per-rank summaries
(row count, order-independent digest, work counter, elapsed time) -- a
gather of a few numbers, not a data-path collective.
"""

from __future__ import annotations

MASK64 = (1 << 64) - 1


def rank_batches(n_batches: int, first_step: int, steps: int, world: int, rank: int) -> list[int]:
    """Batch indices rank `rank` of `world` evaluates in steps
    first_step .. first_step + steps - 1: step s covers batches
    s * world .. s * world + world - 1 (mod n_batches), one per rank."""
    if not 0 <= rank < world or n_batches <= 0:
        raise ValueError("bad rank, world or batch count")
    return [(s * world + rank) % n_batches for s in range(first_step, first_step + steps)]


def combine(parts: list[dict]) -> dict:
    """Whole-job summary from per-rank summaries: counts and work add, the
    digest adds (mod 2^64) and xors, elapsed time is the slowest rank's."""
    out = {"rows": 0, "digest_sum": 0, "digest_xor": 0, "work": 0, "ms": 0.0}
    for p in parts:
        out["rows"] += int(p["rows"])
        out["digest_sum"] = (out["digest_sum"] + int(p["digest_sum"])) & MASK64
        out["digest_xor"] ^= int(p["digest_xor"])
        out["work"] += int(p["work"])
        out["ms"] = max(out["ms"], float(p["ms"]))
    return out


def gather_combine(dist, summary: dict) -> dict:
    """combine() over all ranks of the default process group (every rank
    gets the result)."""
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, summary)
    return combine(parts)
