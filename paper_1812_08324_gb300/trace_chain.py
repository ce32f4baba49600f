"""Critical chain of a traced executor schedule.

    HM_PIPELINE=0 HM_PHASE_TRACE=1 HM_TRACE_FILE=out/tr \\
        python -m paper_1812_08324_gb300.profile_case --n 65536 --what factor --reps 1
    python -m paper_1812_08324_gb300.trace_chain out/tr.factor.txt out/tr.factor.ops.txt

With HM_PHASE_TRACE=1 every schedule run records per task the CTA, SM and
global-timer stamps (grabbed, producers done, finished), and HM_TRACE_FILE
appends them, one line per task with the op's producers, to
<prefix>.<what>.txt (one "# run" section per run; the last one is read) and
the op shapes to <prefix>.<what>.ops.txt.  This walks back from the op that
finished last along the producer that finished last and splits each step
of that chain into

  dispatch  from the producer's finish to the moment a CTA took the task
            (the task waited behind others in the hand-out order), and
  exec      from then to the task's finish (its own run time),

summed per op kind, plus the kinds and shapes that make up the chain.
Files may be gzip-compressed (.gz).
"""
from __future__ import annotations

import collections
import gzip
import sys

KINDS = {0: "gemm", 1: "lu", 2: "trunc", 3: "copy", 4: "reduce", 5: "rows", 6: "vpart"}


def _open(path: str):
    return gzip.open(path, "rt") if path.endswith(".gz") else open(path)


def read_tasks(path: str):
    """Tasks of the last run: {op: [(grab, ready, finish)]}, {op: producers}."""
    runs = []
    cur = None
    with _open(path) as f:
        for line in f:
            if line.startswith("#"):
                cur = ({}, {})
                runs.append(cur)
                continue
            if cur is None:
                cur = ({}, {})
                runs.append(cur)
            head, _, tail = line.partition(":")
            v = [int(x) for x in head.split()]
            op, grab, ready, fin = v[1], v[6], v[7], v[8]
            cur[0].setdefault(op, []).append((grab, ready, fin))
            cur[1][op] = [int(x) for x in tail.split()]
    return runs[-1]


def read_ops(path: str):
    """{op: (kind, dims...)}"""
    out = {}
    with _open(path) as f:
        for line in f:
            v = [int(x) for x in line.split()]
            out[v[0]] = (v[1],) + tuple(v[2:])
    return out


def chain(tasks, prods):
    fin = {op: max(t[2] for t in ts) for op, ts in tasks.items()}
    t0 = min(min(t[0] for t in ts) for ts in tasks.values())
    op = max(fin, key=fin.get)
    out = [op]
    while True:
        ps = [p for p in prods.get(op, []) if p in fin]
        if not ps:
            break
        op = max(ps, key=fin.get)
        out.append(op)
    out.reverse()
    return out, fin, t0


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) < 2:
        print(__doc__)
        return 2
    tasks, prods = read_tasks(argv[0])
    ops = read_ops(argv[1])
    ch, fin, t0 = chain(tasks, prods)
    span = (max(fin.values()) - t0) / 1e6
    print("span %.2f ms, %d ops, %d tasks; critical chain %d ops" %
          (span, len(tasks), sum(len(v) for v in tasks.values()), len(ch)))
    agg = collections.defaultdict(lambda: [0, 0.0, 0.0])
    shapes = collections.Counter()
    prev = t0
    for op in ch:
        last = max(tasks[op], key=lambda t: t[2])
        kind = KINDS.get(ops.get(op, (-1,))[0], "?")
        a = agg[kind]
        a[0] += 1
        a[1] += max(0, last[0] - prev) / 1e3
        a[2] += (fin[op] - max(last[0], prev)) / 1e3
        shapes[(kind,) + tuple(ops.get(op, ())[1:])] += 1
        prev = fin[op]
    tot_d = sum(a[1] for a in agg.values()) / 1e3
    tot_e = sum(a[2] for a in agg.values()) / 1e3
    print("chain: dispatch %.2f ms, exec %.2f ms" % (tot_d, tot_e))
    print("| kind | ops on chain | dispatch | exec | exec per op |")
    print("|---|---|---|---|---|")
    for k, (n, d, e) in sorted(agg.items(), key=lambda kv: -kv[1][2]):
        print("| %s | %d | %.1f ms | %.1f ms | %.2f us |" % (k, n, d / 1e3, e / 1e3, e / max(n, 1)))
    print("most frequent chain ops (kind, dims):")
    for s, n in shapes.most_common(10):
        print("  ", s, n)
    return 0


if __name__ == "__main__":
    sys.exit(main())
