"""Writes tests/golden/discretisation_counts.txt from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py

Every value is an integer of the discretisation the paper describes: the DOFs of the lowest-order
Nedelec space are the mesh edges (Sec. 2.2), without the boundary edges under the PEC condition
(Eq. 1.4) and with them under the impedance condition (Eq. imp); the subdomain index sets follow
Eq. 3.1 on the overlapping boxes of Sec. 6.1; the coarse space is the same space on a coarse mesh
(Sec. 3.2). Small meshes are enumerated by brute force (unique vertex pairs of the tetrahedra)
and assembled; large ones use the oracle's closed forms, which the small ones pin.
"""
import os

import numpy as np

from oracle.mesh import KuhnMesh, count_all_edges, count_interior_edges, count_closed_box_edges
from oracle import fem, dd

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "discretisation_counts.txt")


def main():
    lines = ["# key value -- integer structure of the discretisation; written by make_golden.py (oracle only)",
             "# edges_n / dofs_pec_n / dofs_imp_n: Sec. 2.2, Eq. 1.4, Eq. imp; nnz_pec_n: K and M share it (Sec. 2.2)",
             "# sub_*: Eq. 3.1 on core boxes + overlap (Sec. 6.1); coarse_dofs_m: Sec. 3.2"]
    for n in (1, 2, 3, 4, 6):  # brute force
        m = KuhnMesh(n)
        mi = KuhnMesh(n, "imp")
        K, _ = fem.assemble_KM(m)
        lines.append(f"edges_{n} {m.edges.shape[0]}")
        lines.append(f"dofs_pec_{n} {m.n_dof}")
        lines.append(f"dofs_imp_{n} {mi.n_dof}")
        lines.append(f"nnz_pec_{n} {K.nnz}")
    for n in (10, 12, 40, 60):  # closed forms
        lines.append(f"dofs_pec_{n} {count_interior_edges(n)}")
        lines.append(f"dofs_imp_{n} {count_all_edges(n)}")
    for n, core, ov in ((10, 5, 1), (40, 5, 1), (60, 5, 1)):
        boxes = dd.subdomain_boxes(n, core, ov)
        sizes = [count_interior_edges(*(hi - lo).tolist()) for lo, hi in boxes]
        closed = [count_closed_box_edges(*(hi - lo).tolist()) for lo, hi in boxes]
        tag = f"{n}_{core}_{ov}"
        lines.append(f"sub_count_{tag} {len(boxes)}")
        lines.append(f"sub_min_pec_{tag} {min(sizes)}")
        lines.append(f"sub_max_pec_{tag} {max(sizes)}")
        lines.append(f"sub_sum_pec_{tag} {int(np.sum(sizes))}")
        lines.append(f"sub_sum_imp_{tag} {int(np.sum(closed))}")
    for m in (3, 5, 10, 12):
        lines.append(f"coarse_dofs_pec_{m} {count_interior_edges(m)}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT} ({len(lines)} lines)")


if __name__ == "__main__":
    main()
