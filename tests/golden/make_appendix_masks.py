"""Cross-check harness for the paper's appendix figure (C + AVX2 code).

The appendix of arXiv 2101.01719 prints a complete C implementation of
block_index / make_mask / add_hash / find_hash.  This script extracts that
figure from the paper's LaTeX source at run time (it is never stored in this
repository), appends a small driver written here, compiles it with
``gcc -mavx2`` and runs it.  It needs the paper source and an x86-64 host with
AVX2; callers skip when either is missing.

Run as a script it (re)writes ``appendix_masks.txt`` beside it: the masks and
block indexes the appendix code produces for a few hand-picked hashes.
"""
from __future__ import annotations

import os
import re
import subprocess
import sys
import tempfile

PAPER = os.environ.get("SBBF_PAPER_TEX")  # path of the paper's source text; no default
HERE = os.path.dirname(os.path.abspath(__file__))

# Driver written for this harness: reads "B n_ins n_q" then n_ins + n_q
# hashes; prints block/mask per inserted hash, the filter words after all
# add_hash calls, then find_hash per query.
_DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
int main(void) {
  unsigned long long B, ni, nq;
  if (scanf("%llu %llu %llu", &B, &ni, &nq) != 3) return 2;
  __m256i *f = (__m256i *)aligned_alloc(32, (size_t)B * 32);
  for (unsigned long long b = 0; b < B; ++b) f[b] = _mm256_setzero_si256();
  for (unsigned long long k = 0; k < ni; ++k) {
    unsigned long long h; if (scanf("%llu", &h) != 1) return 3;
    uint32_t m[8];
    _mm256_storeu_si256((__m256i *)m, make_mask((uint32_t)h));
    printf("%llu", (unsigned long long)block_index(h, (uint32_t)B));
    for (int i = 0; i < 8; ++i) printf(" %08x", m[i]);
    printf("\n");
    add_hash(h, (uint32_t)B, f);
  }
  const uint32_t *w = (const uint32_t *)f;
  for (unsigned long long i = 0; i < B * 8; ++i) printf("%08x\n", w[i]);
  for (unsigned long long k = 0; k < nq; ++k) {
    unsigned long long h; if (scanf("%llu", &h) != 1) return 4;
    printf("%d\n", (int)find_hash(h, (uint32_t)B, f));
  }
  free(f);
  return 0;
}
"""


def available() -> str | None:
    """None when the cross-check can run here, else the reason it cannot."""
    if not PAPER:
        return "paper source not configured (set SBBF_PAPER_TEX)"
    if not os.path.exists(PAPER):
        return "paper source not present"
    try:
        flags = open("/proc/cpuinfo").read()
    except OSError:
        return "no /proc/cpuinfo"
    if " avx2" not in flags:
        return "host has no AVX2"
    return None


def extract_figure() -> str:
    text = open(PAPER).read()
    m = re.search(r"\\begin\{verbatim\}\n(.*?)\\end\{verbatim\}", text, re.S)
    if not m:
        raise RuntimeError("appendix figure not found in paper source")
    return m.group(1)


def build(tmpdir: str) -> str:
    src = os.path.join(tmpdir, "appendix.c")
    exe = os.path.join(tmpdir, "appendix")
    with open(src, "w") as fh:
        fh.write(extract_figure())
        fh.write(_DRIVER)
    subprocess.run(["gcc", "-O1", "-mavx2", "-o", exe, src], check=True,
                   capture_output=True)
    return exe


def run(exe: str, num_blocks: int, inserts, queries):
    """Returns (blocks, masks, filter_words, finds) from the appendix code."""
    inp = "%d %d %d\n" % (num_blocks, len(inserts), len(queries))
    inp += "\n".join(str(int(h)) for h in list(inserts) + list(queries)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True,
                         check=True).stdout.split("\n")
    blocks, masks = [], []
    for line in out[: len(inserts)]:
        parts = line.split()
        blocks.append(int(parts[0]))
        masks.append([int(p, 16) for p in parts[1:]])
    pos = len(inserts)
    words = [int(x, 16) for x in out[pos: pos + 8 * num_blocks]]
    pos += 8 * num_blocks
    finds = [int(x) for x in out[pos: pos + len(queries)]]
    return blocks, masks, words, finds


WORKED = [0x0, 0x1, 0x2, 0x80000000, 0xFFFFFFFF, 0x0123456789ABCDEF,
          0xFFFFFFFFFFFFFFFF, 0xDEADBEEFCAFEF00D]


def main() -> int:
    why = available()
    if why:
        print("cannot run the appendix cross-check:", why, file=sys.stderr)
        return 1
    lines = [
        "# Masks and block indexes computed by the paper's appendix figure",
        "# (arXiv 2101.01719, appendix: block_index, make_mask), compiled with",
        "# gcc -mavx2 on x86-64 by tests/golden/make_appendix_masks.py.",
        "# columns: hash  block_index(B=4096)  block_index(B=1000)  mask lane0..lane7",
    ]
    with tempfile.TemporaryDirectory() as d:
        exe = build(d)
        b4096, masks, _, _ = run(exe, 4096, WORKED, [])
        b1000, _, _, _ = run(exe, 1000, WORKED, [])
    for h, a, b, m in zip(WORKED, b4096, b1000, masks):
        lines.append("%016x %d %d %s" % (h, a, b, " ".join("%08x" % x for x in m)))
    with open(os.path.join(HERE, "appendix_masks.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))
    return 0


if __name__ == "__main__":
    sys.exit(main())
