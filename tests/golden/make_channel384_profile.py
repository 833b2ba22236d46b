"""Write channel384_oracle_profile.txt: the FP64 oracle's mean velocity profile
u_x(y) of the 384^3 body-force channel (omega 1, Lambda 3/16, F = 1e-7 along
x, full-way walls at y = 0 and 383, periodic x and z, start from rest) after
5000 steps -- the verification set-up of the paper's Sec. 2.1 at the
reduced-precision workload's size.

A channel run is bitwise independent of x and z (pinned by
test_oracle_pins.py::test_channel_xz_invariance), so the oracle runs the
2 x 384 x 2 column. Calls nothing but the oracle.

    python tests/golden/make_channel384_profile.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "channel384_oracle_profile.txt")


def compute():
    import oracle
    from paper_1711_11468_gb300 import inputs
    c = inputs.CHANNEL_384
    ny = c["dims"][1]
    dims = (2, ny, 2)
    fl = inputs.channel_flags(*dims)
    f = oracle.run(dims, fl, c["omega"], oracle.omega_minus(c["omega"], c["Lambda"]), c["force"],
                   oracle.init_equilibrium(dims, fl), c["steps"])
    _, u = oracle.macroscopic(dims, fl, c["force"], f)
    return u[0].reshape(2, ny, 2)[0, :, 0]


def main():
    prof = compute()
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle: mean u_x(y) of the 384^3 body-force channel after 5000 steps\n")
        fh.write("# (omega 1, Lambda 3/16, F = 1e-7, full-way walls at y = 0 and 383; Sec. 2.1 set-up).\n")
        fh.write("# Written by make_channel384_profile.py from the oracle's 2 x 384 x 2 column.\n")
        fh.write("# y u_x\n")
        for y, v in enumerate(prof):
            fh.write(f"{y} {float(v).hex()}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
