"""Write log_table.inc: the 256 cells of the FP64 logarithm in
karl_device.cuh (Tang's table-driven method).  Cell j covers mantissas
m in [1 + j/256, 1 + (j+1)/256) with centre c_j = 1 + (j + 0.5)/256; each
entry is (ln c_j, 1/c_j) rounded to double.  Run from this directory:
python gen_log_table.py."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def cells():
    for j in range(256):
        c = 1.0 + (j + 0.5) / 256.0
        yield math.log(c), 1.0 / c


def main():
    lines = ["// generated by gen_log_table.py: {ln c_j, 1/c_j}, c_j = 1 + (j + 0.5)/256"]
    for lc, ic in cells():
        lines.append(f"{{{lc!r}, {ic!r}}},")
    with open(os.path.join(HERE, "log_table.inc"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
