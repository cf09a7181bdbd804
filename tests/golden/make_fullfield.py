"""Write the full-field fixtures: the oracle's exact geodesic field on every vertex of the
full-size terrain and torus workloads (first source of each).

Calls only the CPU oracle (oracle/) and the seeded mesh generators; run from the
repository root with `python tests/golden/make_fullfield.py [name ...]` (about 15 minutes
for the terrain and 30 for the torus on one core; the cases run in parallel processes).
The mesh is not stored: the tests rebuild it with the generator and check its SHA-256
against the one recorded here.  Each distance is stored rounded to the nearest double
with a 36-bit mantissa (relative error at most 2^-37, about 7e-12, far inside the 1e-9
parity bar), as six little-endian bytes per value split into byte planes so that the
compressed file stays small."""
import hashlib
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASES = {
    # name: (workload, source index within the workload's first mesh)
    "terrain512_centre": ("terrain", 0),
    "torus1250x400_src0": ("torus", 0),
}
DROP_BITS = 16   # of the 64-bit pattern: keeps sign, exponent and 36 mantissa bits


def mesh_sha256(m) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(m.vertices, dtype="<f8").tobytes())
    h.update(np.ascontiguousarray(m.faces, dtype="<i4").tobytes())
    return h.hexdigest()


def encode(d: np.ndarray) -> np.ndarray:
    bits = np.ascontiguousarray(d, dtype="<f8").view("<u8")
    q = (bits + np.uint64(1 << (DROP_BITS - 1))) >> np.uint64(DROP_BITS)   # round to nearest
    return np.ascontiguousarray(q.astype("<u8").view(np.uint8).reshape(-1, 8)[:, :6].T)


def decode(planes: np.ndarray) -> np.ndarray:
    n = planes.shape[1]
    b = np.zeros((n, 8), dtype=np.uint8)
    b[:, :6] = planes.T
    return (b.reshape(-1).view("<u8") << np.uint64(DROP_BITS)).view("<f8")


def path_of(name: str) -> str:
    return os.path.join(HERE, name + ".npz")


def load(name: str):
    """(field, source vertex, mesh SHA-256, workload) of a stored full-field fixture."""
    z = np.load(path_of(name))
    return decode(z["planes"]), int(z["source"]), str(z["mesh_sha256"]), str(z["workload"])


def make(name: str) -> str:
    import oracle
    from paper_1305_1293_gb300 import meshgen as mg
    wl, si = CASES[name]
    meshes, srcs = mg.workload(wl, "full")
    m, s = meshes[0], int(srcs[0][si])
    t = time.time()
    d, st = oracle.geodesic(m.vertices, m.faces, s)
    np.savez_compressed(path_of(name), planes=encode(d), source=np.int64(s), mesh_sha256=np.array(mesh_sha256(m)),
                        workload=np.array(wl), oracle_windows=np.int64(st["propagated"]))
    return f"{name}: V={m.nv} F={m.nf} source {s}, {st['propagated']} windows, {time.time() - t:.0f} s"


if __name__ == "__main__":
    import oracle
    oracle.build()
    names = sys.argv[1:] or list(CASES)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for line in pool.imap_unordered(make, names):
            print(line, flush=True)
