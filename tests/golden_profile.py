"""Reader for the profiling-summary fixture and a synthetic event list that
reproduces it (two queues, as in the paper's PRNG example)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "golden", "profile_summary_prng.txt")


def load():
    fx = {"agg": {}, "overlap": {}}
    for line in open(PATH):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        parts = line.split()
        kind = parts[0]
        if kind == "agg":
            fx["agg"][parts[1]] = (float(parts[2]), float(parts[3]))
        elif kind == "overlap":
            fx["overlap"][(parts[1], parts[2])] = float(parts[3])
        else:
            fx[kind] = float(parts[1])
    return fx


def synthetic_events(fx):
    """Events whose sums match the fixture: INIT then RNG on the main queue,
    one READ on the comms queue that the RNG kernel overlaps by the printed
    overlap.  Returns (queue, name, start_s, end_s) tuples."""
    init = fx["agg"]["INIT_KERNEL"][1]
    rng = fx["agg"]["RNG_KERNEL"][1]
    read = fx["agg"]["READ_BUFFER"][1]
    ovl = fx["overlap"][("RNG_KERNEL", "READ_BUFFER")]
    read_start = init
    read_end = read_start + read
    rng_start = read_end - ovl          # starts while the read is running
    return [
        ("Main", "INIT_KERNEL", 0.0, init),
        ("Comms", "READ_BUFFER", read_start, read_end),
        ("Main", "RNG_KERNEL", rng_start, rng_start + rng),
    ]
