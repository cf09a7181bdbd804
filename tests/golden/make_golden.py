"""Write the golden fixtures: small meshes with the exact geodesic field of the CPU oracle.

Calls only the oracle (oracle/) and the seeded mesh generators; run from the repository
root with `python tests/golden/make_golden.py`.  Each fixture is a text file holding the
mesh (vertices, faces), the source and the field, so the tests need no generator."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


import oracle  # noqa: E402
from paper_1305_1293_gb300 import meshgen as mg  # noqa: E402

CASES = [
    ("icosphere2_v0", lambda: mg.icosphere(2, 0.02, seed=11), 0),
    ("terrain12x10_corner", lambda: mg.terrain(12, 10, seed=12), 0),
    ("torus16x8_v5", lambda: mg.torus(16, 8, seed=13), 5),
    ("geosphere4_v7", lambda: mg.geodesic_sphere(4, 0.02, seed=14), 7),
]


def write(name, m, s, d):
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write(f"# exact geodesic field of the sequential CPU oracle (Chen-Han / Xin-Wang), source vertex {s}\n")
        f.write(f"{m.nv} {m.nf} {s}\n")
        for v in m.vertices:
            f.write(f"{float(v[0])!r} {float(v[1])!r} {float(v[2])!r}\n")
        for t in m.faces:
            f.write(f"{int(t[0])} {int(t[1])} {int(t[2])}\n")
        for x in d:
            f.write(f"{float(x)!r}\n")


if __name__ == "__main__":
    oracle.build()
    for name, make, s in CASES:
        m = make()
        d, _ = oracle.geodesic(m.vertices, m.faces, s)
        write(name, m, s, d)
        print(name, m.nv, m.nf, float(d.max()))
