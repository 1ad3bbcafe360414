"""Writes oracle_tables.txt: the FP64 oracle's maximum errors of the paper's manufactured
examples (Section 2.3 / Table 2.1 and Section 3.3 / Table 3.1) for m = 19, 39, ..., 99.
Calls only the oracle and the input generators.  Run from the repository root:
    python tests/golden/make_oracle_tables.py"""
import os
import sys
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

M_VALUES = (19, 39, 59, 79, 99)


def table_2_1(args):
    import polar_inputs as pi
    from oracle import polar_oracle as po
    m, radial = args
    p = pi.paper_parabolic_e1(m, radial=radial)
    U = po.run(p)
    return "2.1", m, radial, po.max_error(U, p.exact(p.t[-1]), include_origin=True)


def table_3_1(args):
    import polar_inputs as pi
    from oracle import polar_oracle as po
    m, column = args
    p = pi.paper_continuity_e3(m, radial_adaptive=(column == "uniform_adaptation"))
    U = po.run(p)
    return "3.1", m, column, po.max_error(U, p.exact(p.t[-1]), include_origin=False)


def main():
    jobs = ([(table_2_1, (m, r)) for m in M_VALUES for r in ("sine", "uniform", "zhang")] +
            [(table_3_1, (m, c)) for m in M_VALUES
             for c in ("uniform_adaptation", "radius_non_adaptation")])
    with ProcessPoolExecutor() as ex:
        rows = [f.result() for f in [ex.submit(fn, a) for fn, a in jobs]]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tables.txt")
    with open(out, "w") as f:
        f.write("# Maximum errors at t = 0.1 of the paper's manufactured examples computed by the\n"
                "# FP64 oracle (written by make_oracle_tables.py).  Table 2.1 (Section 2.3): origin\n"
                "# included; columns sine = stretch (2.4), uniform = uniform radial mesh, zhang =\n"
                "# stretch (2.13).  Table 3.1 (Section 3.3): non-origin nodes.\n"
                "# table m column maxerr\n")
        for t, m, c, e in rows:
            f.write(f"{t} {m} {c} {e:.15e}\n")
    print(out)


if __name__ == "__main__":
    main()
