"""Write the full-field fixtures: the oracle's exact geodesic field on every vertex of the
full-size terrain and torus workloads (first source of each).

Calls only the CPU oracle (oracle/) and the seeded mesh generators; run from the
repository root with `python tests/golden/make_fullfield.py [name ...]` (about 15 minutes
for the terrain and 30 for the torus on one core; the cases run in parallel processes).
The mesh is not stored: the tests rebuild it with the generator and check it against
what is recorded here: the SHA-256 of the faces (integers, identical on every machine)
and every 97th vertex (the generator's sines and cosines come from the platform's math
library, which may round differently by an ulp; a coordinate perturbation of that size
moves a distance by far less than the 1e-9 parity bar).  Each distance is stored rounded to the nearest double
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


PROBE_STRIDE = 97


def faces_sha256(m) -> str:
    return hashlib.sha256(np.ascontiguousarray(m.faces, dtype="<i4").tobytes()).hexdigest()


def vertex_probe(m) -> np.ndarray:
    return np.ascontiguousarray(m.vertices[::PROBE_STRIDE], dtype=np.float64)


def same_mesh(m, faces_sha: str, probe: np.ndarray) -> bool:
    """The generator's mesh is the one the field was computed on, up to an ulp-level
    difference of the platform's math library in the coordinates."""
    p = vertex_probe(m)
    return faces_sha256(m) == faces_sha and p.shape == probe.shape and bool(
        np.all(np.abs(p - probe) <= 1e-13 * np.maximum(1.0, np.abs(probe))))


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
    """(field, source vertex, faces SHA-256, vertex probe, workload) of a stored fixture."""
    z = np.load(path_of(name))
    return decode(z["planes"]), int(z["source"]), str(z["faces_sha256"]), z["vertex_probe"], str(z["workload"])


def make(name: str) -> str:
    import oracle
    from paper_1305_1293_gb300 import meshgen as mg
    wl, si = CASES[name]
    meshes, srcs = mg.workload(wl, "full")
    m, s = meshes[0], int(srcs[0][si])
    t = time.time()
    d, st = oracle.geodesic(m.vertices, m.faces, s)
    np.savez_compressed(path_of(name), planes=encode(d), source=np.int64(s), faces_sha256=np.array(faces_sha256(m)),
                        vertex_probe=vertex_probe(m), workload=np.array(wl), oracle_windows=np.int64(st["propagated"]))
    return f"{name}: V={m.nv} F={m.nf} source {s}, {st['propagated']} windows, {time.time() - t:.0f} s"


if __name__ == "__main__":
    import oracle
    oracle.build()
    names = sys.argv[1:] or list(CASES)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for line in pool.imap_unordered(make, names):
            print(line, flush=True)
