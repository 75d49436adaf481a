// Event profiler (Section 3.3 of the cf4ocl paper) and its text summary
// (the layout of the paper's profiling-summary figure, Section 4.1).
//
// Events are (queue, name, start, end) intervals in seconds.  The analysis
// gives, per event name, the summed duration and its share of the total;
// per ordered pair of names, the summed overlap of events on different
// queues (pair = event that started later, event already running); the
// effective time = total - overlaps; and the device share = effective /
// elapsed wall time.  Overlaps are found with one sweep over the events in
// start order, keeping the set of events still running.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

struct rng_prof {
  struct Event {
    std::string queue, name;
    double start, end;
  };
  struct Agg {
    std::string name;
    double abs_s, rel_pct;
  };
  struct Overlap {
    std::string first, second;
    double dur;
  };
  std::vector<Event> events;
  double elapsed = 0.0;
  bool calculated = false;
  std::vector<Agg> aggs;
  std::vector<Overlap> overlaps;
  double total = 0.0, overlap_total = 0.0, effective = 0.0;
  std::string summary;
};

namespace rngi {
// Profilers owned by a generator are not separate library objects: they are
// created and destroyed with it and are not counted by rng_live_objects().
rng_prof *prof_create_owned() { return new (std::nothrow) rng_prof(); }
void prof_destroy_owned(rng_prof *p) { delete p; }
void prof_clear(rng_prof *p) {
  p->events.clear();
  p->calculated = false;
  p->elapsed = 0.0;
}
void prof_add(rng_prof *p, const char *queue, const char *name, double s, double e) {
  p->events.push_back({queue, name, s, e});
  p->calculated = false;
}
}  // namespace rngi

extern "C" {

rng_prof *rng_prof_new(void) {
  rng_prof *p = new (std::nothrow) rng_prof();
  if (p) rngi::live_inc();
  return p;
}

void rng_prof_destroy(rng_prof *p) {
  if (!p) return;
  delete p;
  rngi::live_dec();
}

int rng_prof_add(rng_prof *p, const char *queue, const char *name, double start_s, double end_s) {
  if (!p || !queue || !name || !(end_s >= start_s)) return RNG_EINVAL;
  rngi::prof_add(p, queue, name, start_s, end_s);
  return RNG_OK;
}

int rng_prof_set_elapsed(rng_prof *p, double elapsed_s) {
  if (!p || elapsed_s < 0) return RNG_EINVAL;
  p->elapsed = elapsed_s;
  p->calculated = false;
  return RNG_OK;
}

int rng_prof_calc(rng_prof *p, rng_err **err) {
  if (!p) return rngi::fail(err, RNG_EINVAL, "rng_prof_calc: NULL profiler");
  std::map<std::string, double> agg;
  double total = 0.0;
  for (const auto &e : p->events) {
    agg[e.name] += e.end - e.start;
    total += e.end - e.start;
  }
  p->aggs.clear();
  for (const auto &kv : agg)
    p->aggs.push_back({kv.first, kv.second, total > 0 ? 100.0 * kv.second / total : 0.0});

  // Sweep in start order (index breaks ties, so of two events starting
  // together the later-added one counts as the later starter).
  std::vector<size_t> order(p->events.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return p->events[a].start < p->events[b].start;
  });
  std::map<std::pair<std::string, std::string>, double> ovl;
  std::vector<size_t> running;
  for (size_t idx : order) {
    const auto &e = p->events[idx];
    running.erase(std::remove_if(running.begin(), running.end(),
                                 [&](size_t r) { return p->events[r].end <= e.start; }),
                  running.end());
    for (size_t r : running) {
      const auto &o = p->events[r];
      if (o.queue == e.queue) continue;
      const double len = std::min(o.end, e.end) - e.start;
      if (len > 0) ovl[{e.name, o.name}] += len;
    }
    running.push_back(idx);
  }
  p->overlaps.clear();
  double ovl_total = 0.0;
  for (const auto &kv : ovl) {
    p->overlaps.push_back({kv.first.first, kv.first.second, kv.second});
    ovl_total += kv.second;
  }
  p->total = total;
  p->overlap_total = ovl_total;
  p->effective = total - ovl_total;
  p->calculated = true;
  return RNG_OK;
}

size_t rng_prof_num_aggregates(const rng_prof *p) { return p ? p->aggs.size() : 0; }

int rng_prof_aggregate(const rng_prof *p, size_t index, const char **name, double *abs_s,
                       double *rel_pct) {
  if (!p || index >= p->aggs.size()) return RNG_EINVAL;
  if (name) *name = p->aggs[index].name.c_str();
  if (abs_s) *abs_s = p->aggs[index].abs_s;
  if (rel_pct) *rel_pct = p->aggs[index].rel_pct;
  return RNG_OK;
}

size_t rng_prof_num_overlaps(const rng_prof *p) { return p ? p->overlaps.size() : 0; }

int rng_prof_overlap(const rng_prof *p, size_t index, const char **name1, const char **name2,
                     double *duration_s) {
  if (!p || index >= p->overlaps.size()) return RNG_EINVAL;
  if (name1) *name1 = p->overlaps[index].first.c_str();
  if (name2) *name2 = p->overlaps[index].second.c_str();
  if (duration_s) *duration_s = p->overlaps[index].dur;
  return RNG_OK;
}

double rng_prof_total(const rng_prof *p) { return p ? p->total : 0.0; }
double rng_prof_effective(const rng_prof *p) { return p ? p->effective : 0.0; }
double rng_prof_elapsed(const rng_prof *p) { return p ? p->elapsed : 0.0; }

const char *rng_prof_summary(rng_prof *p, int agg_sort, int ovl_sort) {
  if (!p) return nullptr;
  if (!p->calculated) rng_prof_calc(p, nullptr);
  std::vector<rng_prof::Agg> aggs = p->aggs;
  const bool adesc = (agg_sort & RNG_PROF_SORT_DESC) != 0;
  if ((agg_sort & 0xf) == RNG_PROF_SORT_TIME)
    std::stable_sort(aggs.begin(), aggs.end(), [&](const rng_prof::Agg &a, const rng_prof::Agg &b) {
      return adesc ? a.abs_s > b.abs_s : a.abs_s < b.abs_s;
    });
  else
    std::stable_sort(aggs.begin(), aggs.end(), [&](const rng_prof::Agg &a, const rng_prof::Agg &b) {
      return adesc ? a.name > b.name : a.name < b.name;
    });
  std::vector<rng_prof::Overlap> ovs = p->overlaps;
  const bool odesc = (ovl_sort & RNG_PROF_SORT_DESC) != 0;
  if ((ovl_sort & 0xf) == RNG_PROF_SORT_TIME)
    std::stable_sort(ovs.begin(), ovs.end(),
                     [&](const rng_prof::Overlap &a, const rng_prof::Overlap &b) {
                       return odesc ? a.dur > b.dur : a.dur < b.dur;
                     });
  else
    std::stable_sort(ovs.begin(), ovs.end(),
                     [&](const rng_prof::Overlap &a, const rng_prof::Overlap &b) {
                       auto ka = std::make_pair(a.first, a.second);
                       auto kb = std::make_pair(b.first, b.second);
                       return odesc ? ka > kb : ka < kb;
                     });
  std::string s;
  char line[256];
  const char *rule = "   ------------------------------------------------------------------\n";
  s += " Aggregate times by event  :\n";
  s += rule;
  s += "   | Event name                     | Rel. time (%) | Abs. time (s) |\n";
  s += rule;
  for (const auto &a : aggs) {
    snprintf(line, sizeof line, "   | %-30.30s | %13.4f | %13.4e |\n", a.name.c_str(), a.rel_pct,
             a.abs_s);
    s += line;
  }
  s += rule;
  snprintf(line, sizeof line, "                                    |         Total | %13.4e |\n",
           p->total);
  s += line;
  s += "                                    ---------------------------------\n";
  if (!ovs.empty()) {
    s += " Event overlaps            :\n";
    s += rule;
    s += "   | Event 1                | Event 2                | Overlap (s)  |\n";
    s += rule;
    for (const auto &o : ovs) {
      snprintf(line, sizeof line, "   | %-22.22s | %-22.22s | %12.4e |\n", o.first.c_str(),
               o.second.c_str(), o.dur);
      s += line;
    }
    s += rule;
    snprintf(line, sizeof line, "                            |                  Total | %12.4e |\n",
             p->overlap_total);
    s += line;
    s += "                            -----------------------------------------\n";
  }
  snprintf(line, sizeof line, " Tot. of all events (eff.) : %es\n", p->effective);
  s += line;
  snprintf(line, sizeof line, " Total elapsed time        : %es\n", p->elapsed);
  s += line;
  const double dev = p->elapsed > 0 ? 100.0 * p->effective / p->elapsed : 0.0;
  snprintf(line, sizeof line, " Time spent in device      : %.2f%%\n", dev);
  s += line;
  snprintf(line, sizeof line, " Time spent in host        : %.2f%%\n", 100.0 - dev);
  s += line;
  p->summary = s;
  return p->summary.c_str();
}

int rng_prof_export(rng_prof *p, const char *path, rng_err **err) {
  if (!p || !path) return rngi::fail(err, RNG_EINVAL, "rng_prof_export: NULL argument");
  std::vector<size_t> order(p->events.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return p->events[a].start < p->events[b].start;
  });
  const double t0 = order.empty() ? 0.0 : p->events[order[0]].start;
  FILE *f = fopen(path, "w");
  if (!f) return rngi::fail(err, RNG_EINVAL, "rng_prof_export: cannot open %s", path);
  for (size_t i : order) {
    const auto &e = p->events[i];
    fprintf(f, "%s\t%.0f\t%.0f\t%s\n", e.queue.c_str(), (e.start - t0) * 1e9, (e.end - t0) * 1e9,
            e.name.c_str());
  }
  const bool ok = fclose(f) == 0;
  return ok ? RNG_OK : rngi::fail(err, RNG_EINVAL, "rng_prof_export: write to %s failed", path);
}

}  // extern "C"
