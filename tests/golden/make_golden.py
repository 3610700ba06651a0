"""Writes the oracle regression fixtures in this folder (calls only oracle/ and synth/).

The paper prints no worked k-mer example, so these fixtures are not the paper's
numbers: they freeze the oracle's output on small seeded inputs so that a later
change to the oracle's arithmetic shows up as a diff.  Regenerate with
``python tests/golden/make_golden.py`` and justify the change in the commit.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402

# the single-genome recipe shrunk to a 600 bp genome at 30x (120 reads x 150 bp)
SMALL = synth.SINGLE_GENOME.scaled(120, genome_len_min=600, genome_len_max=600, name="single-genome-600bp")
CASES = [
    # (file, recipe, n_reads, params)
    ("single_genome_600bp_k21.txt", SMALL, 120, oracle.Params(k=21, min_count=2)),
    ("single_genome_600bp_k33_static.txt", SMALL, 120, oracle.Params(k=33, min_count=2, ext_mode=1, t_ext=2)),
]


def render(res: oracle.Result) -> str:
    lines = [f"# windows={res.windows} distinct={res.distinct} survivors={len(res)}"]
    for i in range(len(res)):
        ext = " ".join(str(int(x)) for x in res.ext[i])
        lines.append(f"{res.keys[i].decode()} {int(res.count[i])} {ext} {int(res.cls[i, 0])} {int(res.cls[i, 1])}")
    return "\n".join(lines) + "\n"


def compute(recipe, n_reads, params):
    rs = synth.generate(recipe.scaled(n_reads))
    return oracle.run(rs.bases, rs.quals, rs.offsets, params)


if __name__ == "__main__":
    for name, recipe, n, p in CASES:
        with open(os.path.join(HERE, name), "w") as f:
            f.write(f"# oracle output, recipe={recipe.name} first {n} reads, params={p}\n")
            f.write(render(compute(recipe, n, p)))
        print("wrote", name)
