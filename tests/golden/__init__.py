"""Reader for the golden fixtures (values printed in the paper)."""
from __future__ import annotations

import os
from collections import defaultdict

_DIR = os.path.dirname(os.path.abspath(__file__))


def _num(tok: str) -> int:
    return int(tok, 16) if tok.lower().startswith(("0x", "-0x")) else int(tok)


def paper_examples() -> dict:
    """``key -> list of lines``; each line is a list of tokens."""
    out = defaultdict(list)
    with open(os.path.join(_DIR, "paper_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(":")
            out[key.strip()].append(rest.split())
    return dict(out)


def ints(key: str) -> list:
    return [_num(t) for t in paper_examples()[key][0]]


def text(key: str) -> str:
    return paper_examples()[key][0][0]


def rows(key: str) -> list:
    return [[_num(t) for t in r] for r in paper_examples()[key]]
