"""Writes the stored fixtures under tests/golden/.

Run from the repository root: python tests/golden/make_golden.py
It calls only the seeded generators (and, for values, only oracle/).
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2601_02826_gb300 import synth  # noqa: E402


def main():
    a = synth.tiny_geno(123, 50, 20)
    h = hashlib.sha256(a.geno.tobytes()).hexdigest()[:16]
    with open(os.path.join(HERE, "tiny_geno_123_50x20.sha256"), "w") as f:
        f.write(f"{h}  sha256[:16] of synth.tiny_geno(123, 50, 20).geno (int8, SNP-major, ld=64)\n")


if __name__ == "__main__":
    main()
