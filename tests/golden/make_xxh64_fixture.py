"""Write xxh64_known_answers.txt: XXH64 of seeded byte strings computed by the
reference xxHash library (libxxhash, the implementation published with the
xxHash specification), so the oracle's XXH64 stays pinned on machines where
the library is not installed.

Each line: <length> <seed> <hash, 16 hex digits> <input bytes as hex>.
Inputs: every length 0..72 (the 32-byte stripe loop, the 8-, 4- and 1-byte
tails), a few longer ones, and the 8 little-endian bytes of 64-bit term codes
(the hashed form of a term); seeds 0, 1, 2 (hash indices) and two large ones.

Run once with libxxhash present:  python tests/golden/make_xxh64_fixture.py
"""
import ctypes
import ctypes.util
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "xxh64_known_answers.txt")
SEEDS = (0, 1, 2, 0xFFFFFFFFFFFFFFFF, 12345678901234567)


def libxxhash():
    for name in ("libxxhash.so.0", "libxxhash.so", ctypes.util.find_library("xxhash")):
        if not name:
            continue
        try:
            lib = ctypes.CDLL(name)
        except OSError:
            continue
        lib.XXH64.restype = ctypes.c_uint64
        lib.XXH64.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
        return lib
    return None


def inputs():
    rng = np.random.default_rng(20190523)
    for n in list(range(0, 73)) + [96, 127, 128, 255, 1000]:
        yield rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
    for code in (0, 1, 0x0123456789ABCDEF, (1 << 62) - 1, 0xFFFFFFFFFFFFFFFF, 0x3FFFFFFFFFFFFFFF,
                 int(rng.integers(0, 1 << 62, dtype=np.uint64))):
        yield int(code).to_bytes(8, "little")


def main():
    lib = libxxhash()
    if lib is None:
        sys.exit("libxxhash is required to write the fixture")
    lines = []
    for data in inputs():
        buf = ctypes.create_string_buffer(data, max(len(data), 1))
        for seed in SEEDS:
            lines.append(f"{len(data)} {seed} {lib.XXH64(buf, len(data), seed):016x} {data.hex()}")
    with open(OUT, "w") as f:
        f.write("# XXH64 known answers from libxxhash (tests/golden/make_xxh64_fixture.py)\n")
        f.write("# length seed hash-hex input-hex\n")
        f.write("\n".join(lines) + "\n")
    print(f"{len(lines)} answers -> {OUT}")


if __name__ == "__main__":
    main()
