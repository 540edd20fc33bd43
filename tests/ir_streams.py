"""Builders of the paper's example task streams as oracle IR objects (tests only)."""
import os

from oracle.ir import Arg, IDENTITY, NonePart, Task, Tiling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def fig1_stream(N=4, tiles=(2, 2)):
    """The stencil iteration of Fig. 1c as IR tasks over an (N+2)^2 grid.

    Returns (tasks, names, root boxes, app_held) with store ids: 0 = grid and
    one id per array temporary; views are boxes of the grid (Fig. 1a)."""
    th, tw = N // tiles[0], N // tiles[1]
    grid = 0
    views = {"center": (1, 1), "north": (0, 1), "east": (1, 2), "west": (1, 0), "south": (2, 1)}
    ids = {"grid": 0}
    boxes = {0: ((0, 0), (N + 2, N + 2))}

    def vpart(name):
        o = views[name]
        box = (o, (o[0] + N, o[1] + N))
        return grid, Tiling((th, tw), o, IDENTITY, box)

    def apart(name):
        if name not in ids:
            ids[name] = len(ids)
            boxes[ids[name]] = ((0, 0), (N, N))
        return ids[name], Tiling((th, tw), (0, 0), IDENTITY, ((0, 0), (N, N)))

    def part(name):
        return vpart(name) if name in views else apart(name)

    tasks = []
    for row in read_golden("fig1_stencil_stream.txt"):
        if row[0] != "task":
            continue
        name, out, ins = row[1], row[2], row[3:]
        args = []
        for i in ins:
            try:
                float(i)
                continue  # immediate
            except ValueError:
                s, p = part(i)
                args.append(Arg(s, p, "R"))
        s, p = part(out)
        args.append(Arg(s, p, "W"))
        tasks.append(Task(name, tiles, args))
    return tasks, ids, boxes, {grid}


def temp_elim_stream(n=8):
    """Fig. 6b over 1-D stores of n elements, launch domain (2,)."""
    ids = {}
    boxes = {}

    def full(name):
        if name not in ids:
            ids[name] = len(ids)
            boxes[ids[name]] = ((0,), (n,))
        return ids[name], Tiling((n // 2,), (0,), IDENTITY, ((0,), (n,)))

    tasks = []
    app = set()
    for row in read_golden("temp_elim_example.txt"):
        if row[0] == "task":
            name, out, ins = row[1], row[2], row[3:]
            args = []
            for i in ins:
                try:
                    float(i)
                    continue
                except ValueError:
                    pass
                if i == "whalf":
                    s, _ = full("w")
                    args.append(Arg(s, Tiling((n // 4,), (n // 2,), IDENTITY, ((n // 2,), (n,))), "R"))
                else:
                    s, p = full(i)
                    args.append(Arg(s, p, "R"))
            if name == "NORM":
                if out not in ids:
                    ids[out] = len(ids)
                    boxes[ids[out]] = ((), ())
                args.append(Arg(ids[out], NonePart(((), ())), "Rd"))
            else:
                s, p = full(out)
                args.append(Arg(s, p, "W"))
            tasks.append(Task(name, (2,), args))
        elif row[0] == "apphold":
            app = {ids[x] for x in row[1:]}
    return tasks, ids, boxes, app


def memo_streams():
    """Fig. 7a streams keyed by id; every arg uses one partition and domain."""
    part = Tiling((4,), (0,), IDENTITY, ((0,), (8,)))
    streams = {}
    cur = None
    canon = {}
    for row in read_golden("memo_streams.txt"):
        if row[0] == "stream":
            cur = row[1]
            streams[cur] = []
        elif row[0] == "task":
            args = []
            for a in row[2:]:
                s, p = a.split(":")
                args.append(Arg(int(s[1:]), part, p))
            streams[cur].append(Task(row[1], (2,), args))
        elif row[0] == "canonical":
            tasks = " ".join(row[2:]).split(";")
            form = []
            for t in tasks:
                f = t.split()
                form.append((f[0], tuple((int(x.split(":")[0]), x.split(":")[1]) for x in f[1:])))
            canon[row[1]] = form
    return streams, canon
