"""Command-line generator in the form of the paper's example program
(Section 5): ``python -m paper_1609_01257_gb300 n i [--seed S] [--profile]``
writes i iterations of n 64-bit values as raw binary to stdout (8*n*i bytes,
Eq. 1), e.g. ``python -m paper_1609_01257_gb300 16777216 10000 | consumer``.
With ``--profile`` the profiling summary goes to stderr."""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1609_01257_gb300", description=__doc__)
    ap.add_argument("n", type=int, help="64-bit values per iteration (streams)")
    ap.add_argument("i", type=int, help="iterations")
    ap.add_argument("--seed", type=int, default=0, help="run seed (0: the paper's generator)")
    ap.add_argument("--buffer-bytes", type=int, default=32 << 20, help="size of each device buffer")
    ap.add_argument("--profile", action="store_true", help="print the profiling summary to stderr")
    ap.add_argument("--output-mode", type=int, choices=[0, 1], default=0,
                    help="0: the paper's values (the states); 1: xorshift64* scrambled values")
    args = ap.parse_args(argv)
    from . import Generator
    g = Generator(args.n, args.seed, device_buffer_bytes=args.buffer_bytes, host_path=1,
                  output_mode=args.output_mode)
    sys.stdout.flush()
    g.generate_fd(args.i, sys.stdout.fileno())
    if args.profile:
        sys.stderr.write(g.profile_summary())
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
